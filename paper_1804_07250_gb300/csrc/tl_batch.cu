// Batched chains: one launch advances every tile of every chain by R sweeps.
//
// Many independent chains of uneven size (the batched workload of Sec. 4's
// sampling experiments) are cut into row stripes ("tiles").  A CTA takes
// tiles from a work list ordered largest first, loads a tile plus a halo of
// passes * R rows from the chain's source buffer into shared memory, runs the
// R sweeps there with the exact region shrinking one row per pass, and writes
// only the tile's own rows to the destination buffer.  Because tiles of one
// chain run concurrently within a launch, a launch reads one buffer and
// writes the other; consecutive launches alternate.  Sweep indices come from
// a per-chain device counter, so a block of launches captured in a CUDA graph
// can be replayed: the graph ends with a kernel that advances the counters.
#include "tl_device.cuh"

#include <cstdint>

namespace tl {

// Bulk asynchronous copies (the copy engine of sm_90+, cp.async.bulk) between
// global and shared memory, completed through an mbarrier (loads) or a bulk
// group (stores).  Addresses 16-byte aligned, sizes multiples of 16 bytes.
TL_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
TL_DEV void mbar_init(unsigned long long* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
TL_DEV void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
TL_DEV bool mbar_try_wait(unsigned long long* bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
TL_DEV uint64_t batch_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of `parity` to complete, at most about two seconds.
TL_DEV bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity)
{
    const uint64_t t0 = batch_globaltimer();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 0 && batch_globaltimer() - t0 > 2000000000ull) return false;
    }
}
TL_DEV void bulk_store(void* dst, const void* src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
TL_DEV void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
TL_DEV void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
TL_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int LAT, int TK>
TL_DEV void tile_passes(const BatchChain& ch, uint32_t* srow0, int slo, int shi, bool bot, bool top, uint32_t sweep0,
                        int R)
{
    const Geom& g = ch.g;
    const int64_t RW = g.row_words;
    const int passes = g.passes;
    int i = 0;
    for (int r = 0; r < R; ++r) {
        const uint32_t sweep = sweep0 + (uint32_t)r;
        for (int p = 0; p < passes; ++p, ++i) {
            const int vlo = bot ? -1 : slo + i;
            const int vhi = top ? g.H + 1 : shi - i;
            int a, nrows, step;
            if (LAT == LAT_SIXV) {
                a = vlo > 1 ? vlo : 1;
                const int last = (vhi - 2) < (g.N - 1) ? (vhi - 2) : (g.N - 1);
                if ((a & 1) != sixv_py((uint32_t)p)) ++a;
                step = 2;
                nrows = last >= a ? (last - a) / 2 + 1 : 0;
            } else {
                a = (vlo + 1) > 0 ? (vlo + 1) : 0;
                const int b = vhi < g.H ? vhi : g.H;
                step = 1;
                nrows = b > a ? b - a : 0;
            }
            const int items = nrows * g.Kg;
            for (int it = threadIdx.x; it < items; it += blockDim.x) {
                const int ri = it / g.Kg, m = it - ri * g.Kg;
                const int y = a + ri * step;
                const int2 gr = ch.grange[y];
                if (m < gr.x || m >= gr.y) continue;
                const uint32_t grp = (uint32_t)(((LAT == LAT_SIXV) ? (y >> 1) : y) * g.Kg + m);
                const RndPhilox rnd{grp, sweep, (uint32_t)p, ch.rng};
                group_update<LAT, TK>(srow0 + (int64_t)y * RW, RW, g, y, m, (uint32_t)p, rnd, ch.th);
            }
            __syncthreads();
        }
    }
}

// NT threads per tile: a thread takes every NT-th 128-face group of a pass
// (the faces per thread the autotuner picks).  256 threads: three CTAs per
// SM (at most 85 registers a thread): the passes of a tile are separated by
// barriers, and a third resident tile hides them better than the registers
// spilled to L1 cost (two CTAs at 124 registers measured 9% slower, four at
// 64 registers no faster).  128 threads: six CTAs per SM at the same
// registers, twice the faces per thread, as many tiles as shared memory
// holds.
template <int NT>
__global__ void __launch_bounds__(NT, NT == 128 ? 6 : 3) batch_kernel(const BatchChain* __restrict__ chains,
                                                                    const BatchTile* __restrict__ tiles, int ntiles,
                                                                    int R, uint32_t sweep_off, int src,
                                                                    unsigned int* cursor, int* __restrict__ status)
{
    extern __shared__ uint4 smem4[];
    __shared__ int s_tile;
    __shared__ __align__(8) unsigned long long s_bar;
    uint32_t* sm = reinterpret_cast<uint32_t*>(smem4);
    if (threadIdx.x == 0) mbar_init(&s_bar, 1);
    __syncthreads();
    uint32_t parity = 0;
    for (;;) {
        // a raised status word (a wait that gave up elsewhere, or raised by
        // the host) stops the block before it issues another copy
        if (threadIdx.x == 0) s_tile = *(volatile int*)status ? ntiles : (int)atomicAdd(cursor, 1u);
        __syncthreads();
        const int t = s_tile;
        __syncthreads();
        if (t >= ntiles) break;
        const BatchTile tile = tiles[t];
        const BatchChain& ch = chains[tile.chain];
        const Geom& g = ch.g;
        const int64_t RW = g.row_words;
        const int halo = g.passes * R;
        const bool bot = tile.lo == 0, top = tile.hi == g.H;
        const int slo = bot ? -1 : (tile.lo - halo > -1 ? tile.lo - halo : -1);
        const int shi = top ? g.H + 1 : (tile.hi + halo < g.H + 1 ? tile.hi + halo : g.H + 1);
        // a halo clamped at a pad row is exact from then on
        const bool bot_x = slo == -1, top_x = shi == g.H + 1;
        const uint32_t* srcp = ch.rows[src] + RW;   // global row 0
        uint32_t* dstp = ch.rows[src ^ 1] + RW;
#ifdef TL_DEBUG
        {
            // the tile and its halo rows fit the block's shared memory
            uint32_t dyn;
            asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
            if (!TL_IN((int64_t)(shi - slo) * RW * 4 - 1, (int64_t)dyn, 301)) continue;
        }
#endif
        // the tile and its halo rows are contiguous: one bulk copy into shared
        // memory (rows are whole 16-byte units, buffers 256-byte aligned)
        if (threadIdx.x == 0) bulk_load(sm, srcp + (int64_t)slo * RW, (uint32_t)((int64_t)(shi - slo) * RW * 4), &s_bar);
        const int arrived = __syncthreads_and(mbar_wait_bounded(&s_bar, parity) ? 1 : 0);
        parity ^= 1u;
        if (!arrived) {
            // the copy did not complete in two seconds: report, give the copy
            // one more bounded wait so that nothing is left writing this
            // block's shared memory, and stop (every thread of the block
            // takes this branch together)
            if (threadIdx.x == 0) {
                atomicExch(status, 1);
                mbar_wait_bounded(&s_bar, parity ^ 1u);
            }
            __syncthreads();
            return;
        }
        const uint32_t sweep0 = *ch.sweep_base + sweep_off;
        uint32_t* srow0 = sm - (int64_t)slo * RW;
        if (g.lattice == LAT_DOMINO) {
            if (ch.th.kind == THR_SITE) tile_passes<LAT_DOMINO, THR_SITE>(ch, srow0, slo, shi, bot_x, top_x, sweep0, R);
            else tile_passes<LAT_DOMINO, THR_SCALAR>(ch, srow0, slo, shi, bot_x, top_x, sweep0, R);
        } else if (g.lattice == LAT_LOZENGE) {
            if (ch.th.kind == THR_SITE) tile_passes<LAT_LOZENGE, THR_SITE>(ch, srow0, slo, shi, bot_x, top_x, sweep0, R);
            else tile_passes<LAT_LOZENGE, THR_SCALAR>(ch, srow0, slo, shi, bot_x, top_x, sweep0, R);
        } else {
            tile_passes<LAT_SIXV, THR_TABLE>(ch, srow0, slo, shi, bot_x, top_x, sweep0, R);
        }
        // the tile's own rows back in one bulk copy; shared memory is reused
        // by the next tile once the copy has read it
        fence_proxy_async();
        __syncthreads();
        if (threadIdx.x == 0) {
            bulk_store(dstp + (int64_t)tile.lo * RW, srow0 + (int64_t)tile.lo * RW,
                       (uint32_t)((int64_t)(tile.hi - tile.lo) * RW * 4));
            bulk_wait_read();
        }
        // the pad rows of the destination stay zero: they are never written
        __syncthreads();
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

__global__ void batch_advance_kernel(const BatchChain* __restrict__ chains, int nchains, uint32_t k,
                                     unsigned int* cursors, int ncursors)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nchains; i += gridDim.x * blockDim.x)
        *chains[i].sweep_base += k;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncursors; i += gridDim.x * blockDim.x) cursors[i] = 0u;
}

static const void* batch_pick(int threads)
{
    return threads == 128 ? reinterpret_cast<const void*>(&batch_kernel<128>)
                          : reinterpret_cast<const void*>(&batch_kernel<256>);
}

int batch_prepare(size_t smem_bytes, int threads, int* blocks_per_sm)
{
    const void* k = batch_pick(threads);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (int)e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads == 128 ? 128 : 256, smem_bytes);
    if (e != cudaSuccess) cudaGetLastError();
    return (int)e;
}

int launch_batch(const BatchChain* chains, const BatchTile* tiles, int ntiles, int R, uint32_t sweep_off, int src,
                 unsigned int* cursor, int grid, int threads, size_t smem_bytes, int* status, void* stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (threads == 128)
        batch_kernel<128><<<grid, 128, smem_bytes, st>>>(chains, tiles, ntiles, R, sweep_off, src, cursor, status);
    else
        batch_kernel<256><<<grid, 256, smem_bytes, st>>>(chains, tiles, ntiles, R, sweep_off, src, cursor, status);
    return (int)cudaGetLastError();
}

int launch_batch_advance(const BatchChain* chains, int nchains, uint32_t k, unsigned int* cursors, int ncursors,
                         void* stream)
{
    const int n = nchains > ncursors ? nchains : ncursors;
    batch_advance_kernel<<<(n + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(chains, nchains, k,
                                                                                             cursors, ncursors);
    return (int)cudaGetLastError();
}

// Per-chain state hash over all tiles (out[chain] must be zeroed).
__global__ void batch_hash_kernel(const BatchChain* __restrict__ chains, const BatchTile* __restrict__ tiles,
                                  int ntiles, int buf, unsigned long long* out)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tile = tiles[t];
        const BatchChain& ch = chains[tile.chain];
        const Geom& g = ch.g;
        const int64_t RW = g.row_words;
        const uint32_t* base = ch.rows[buf] + RW + (int64_t)tile.lo * RW;
        const int nw = (tile.hi - tile.lo) * (int)RW;
        uint64_t acc = 0;
        for (int w = threadIdx.x; w < nw; w += blockDim.x) {
            const uint32_t v = base[w];
            if (!v) continue;
            const int rr = w / (int)RW;
            const int rem = w - rr * (int)RW;
            const int pl = rem / g.K, k = rem - pl * g.K;
            acc += word_hash(v, g, tile.lo + rr, pl, k);
        }
        for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
        if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out + tile.chain, (unsigned long long)acc);
    }
}

int launch_batch_hash(const BatchChain* chains, const BatchTile* tiles, int ntiles, int buf,
                      unsigned long long* out, void* stream)
{
    const int grid = ntiles < 4096 ? ntiles : 4096;
    batch_hash_kernel<<<grid > 0 ? grid : 1, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(chains, tiles, ntiles,
                                                                                             buf, out);
    return (int)cudaGetLastError();
}

// Copy every tile's rows from buffer `from` to the other buffer.
__global__ void batch_copy_kernel(const BatchChain* __restrict__ chains, const BatchTile* __restrict__ tiles,
                                  int ntiles, int from)
{
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const BatchTile tile = tiles[t];
        const BatchChain& ch = chains[tile.chain];
        const int64_t RW = ch.g.row_words;
        const uint4* s4 = reinterpret_cast<const uint4*>(ch.rows[from] + RW + (int64_t)tile.lo * RW);
        uint4* d4 = reinterpret_cast<uint4*>(ch.rows[from ^ 1] + RW + (int64_t)tile.lo * RW);
        const int64_t n4 = (int64_t)(tile.hi - tile.lo) * RW / 4;
        for (int64_t i = threadIdx.x; i < n4; i += blockDim.x) d4[i] = s4[i];
    }
}

int launch_batch_copy(const BatchChain* chains, const BatchTile* tiles, int ntiles, int from, void* stream)
{
    const int grid = ntiles < 4096 ? ntiles : 4096;
    batch_copy_kernel<<<grid > 0 ? grid : 1, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(chains, tiles, ntiles,
                                                                                             from);
    return (int)cudaGetLastError();
}

// This file's debug word (failures, then the id, index and bound of the
// first failed check); cudaErrorNotSupported in the normal build.
int dbg_fetch_batch(unsigned long long* out, bool clear)
{
#ifdef TL_DEBUG
    return tl_dbg_fetch(out, clear);
#else
    (void)out;
    (void)clear;
    return (int)cudaErrorNotSupported;
#endif
}

}  // namespace tl
