// Shared-memory resident multi-sweep kernel (cooperative launch).
//
// The paper launches Rotate and Update once per half-step and moves the
// whole tiling through device memory every time (Sec. 2.2).  Here one launch
// runs many sweeps: each CTA keeps a horizontal stripe of the packed state
// plus `halo` rows above and below it in shared memory.  A pass updates every
// row whose inputs are still exact; because a site only reads edges within
// one row of it, the exact region shrinks by one row at each interior stripe
// edge per pass, so after `halo` passes the CTA still holds its own rows
// exactly.  It then publishes its top and bottom `halo` rows, waits for its
// two neighbours' progress flags (bounded wait), and refreshes its halos.
// State thus crosses the memory system once per `halo` passes and only at
// stripe seams; the rest of the time it stays on chip.
#include "tl_device.cuh"

#include <cstdint>

namespace tl {

struct ResParams {
    uint32_t* rows0;            // global row 0 (after the pad row)
    Geom g;
    const int* stripe_lo;
    int halo;
    uint32_t sweep0, nsweeps;
    DevRng rng;
    ThrView th;
    const int2* grange;
    uint32_t* xbuf;
    unsigned long long* flags;
    int* status;
    unsigned long long* ring;
    uint32_t* counts;
    uint64_t burn;
    uint32_t stride;
    unsigned int epoch;
};

TL_DEV unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
TL_DEV void st_release(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
TL_DEV uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: far beyond any healthy exchange

// Copy `nrows` packed rows (16-byte granules), L2 only on the global side.
TL_DEV void copy_rows_to_global(uint32_t* dst, const uint32_t* src, int64_t words, int tid, int nt)
{
    uint4* d = reinterpret_cast<uint4*>(dst);
    const uint4* s = reinterpret_cast<const uint4*>(src);
    for (int64_t i = tid; i < words / 4; i += nt) __stcg(d + i, s[i]);
}
TL_DEV void copy_rows_from_global(uint32_t* dst, const uint32_t* src, int64_t words, int tid, int nt)
{
    uint4* d = reinterpret_cast<uint4*>(dst);
    const uint4* s = reinterpret_cast<const uint4*>(src);
    for (int64_t i = tid; i < words / 4; i += nt) d[i] = __ldcg(s + i);
}

template <int LAT, int TK>
__global__ void __launch_bounds__(512, 1) resident_kernel(const ResParams P)
{
    extern __shared__ uint4 smem4[];
    __shared__ int s_ok;
    __shared__ unsigned long long s_red[16];
    const Geom& g = P.g;
    const int64_t RW = g.row_words;
    const int c = blockIdx.x, C = gridDim.x;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int lo = P.stripe_lo[c], hi = P.stripe_lo[c + 1];
    const bool bot = (c == 0), top = (c == C - 1);
    const int h = P.halo;
    const int slo = bot ? -1 : lo - h;
    const int shi = top ? g.H + 1 : hi + h;
    uint32_t* sm = reinterpret_cast<uint32_t*>(smem4);
    uint32_t* srow0 = sm - (int64_t)slo * RW;   // srow0 + y * RW is global row y

    copy_rows_from_global(sm, P.rows0 + (int64_t)slo * RW, (int64_t)(shi - slo) * RW, tid, nt);
    __syncthreads();

    const int passes = g.passes;
    const uint64_t total = (uint64_t)P.nsweeps * passes;
    const size_t side_words = (size_t)h * RW;
    uint64_t done = 0;
    int cyc = 0;
    while (done < total) {
        const int hc = (int)((total - done) < (uint64_t)h ? (total - done) : (uint64_t)h);
        for (int i = 1; i <= hc; ++i) {
            const uint64_t pidx = done + (uint64_t)(i - 1);
            const uint32_t sweep = P.sweep0 + (uint32_t)(pidx / passes);
            const uint32_t pass = (uint32_t)(pidx % passes);
            // rows [vlo, vhi) are exact before this pass
            const int vlo = bot ? -1 : slo + (i - 1);
            const int vhi = top ? g.H + 1 : shi - (i - 1);
            int r0, nrows, rstep;
            if (LAT == LAT_SIXV) {
                // face rows Y with vertex rows Y and Y+1 exact, of this class's parity
                int a = vlo > 1 ? vlo : 1;
                const int last = (vhi - 2) < (g.N - 1) ? (vhi - 2) : (g.N - 1);
                if ((a & 1) != sixv_py(pass)) ++a;
                r0 = a;
                rstep = 2;
                nrows = last >= a ? (last - a) / 2 + 1 : 0;
            } else {
                const int a = (vlo + 1) > 0 ? (vlo + 1) : 0;
                const int b = vhi < g.H ? vhi : g.H;
                r0 = a;
                rstep = 1;
                nrows = b > a ? b - a : 0;
            }
            const int items = nrows * g.Kg;
            for (int it = tid; it < items; it += nt) {
                const int ri = it / g.Kg, m = it - ri * g.Kg;
                const int y = r0 + ri * rstep;
                const int2 gr = P.grange[y];
                if (m < gr.x || m >= gr.y) continue;
                const uint32_t grp = (uint32_t)(((LAT == LAT_SIXV) ? (y >> 1) : y) * g.Kg + m);
                group_update<LAT, TK>(srow0 + (int64_t)y * RW, RW, g, y, m, pass, grp, sweep, P.rng, P.th);
            }
            __syncthreads();
            if (pass == (uint32_t)(passes - 1)) {
                // end of a sweep: the owned rows are exact (i <= halo)
                const uint64_t ndone = (uint64_t)sweep + 1;
                const bool sample = P.counts && P.stride && ndone >= P.burn &&
                                    (ndone - P.burn) % P.stride == 0;
                if (P.ring || sample) {
                    const int64_t nw = (int64_t)(hi - lo) * RW;
                    const uint32_t* base = srow0 + (int64_t)lo * RW;
                    uint64_t acc = 0;
                    for (int64_t w = tid; w < nw; w += nt) {
                        const uint32_t v = base[w];
                        if (!v) continue;
                        const int yy = lo + (int)(w / RW);
                        const int rem = (int)(w - (int64_t)(yy - lo) * RW);
                        const int pl = rem / g.K, k = rem - pl * g.K;
                        if (P.ring) acc += word_hash(v, g, yy, pl, k);
                        if (sample) word_count(v, g, yy, pl, k, P.counts);
                    }
                    if (P.ring) {
                        for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
                        if ((tid & 31) == 0) s_red[tid >> 5] = acc;
                        __syncthreads();
                        if (tid == 0) {
                            unsigned long long t = 0;
                            for (int wv = 0; wv < (nt + 31) / 32; ++wv) t += s_red[wv];
                            atomicAdd(P.ring + (sweep - P.sweep0), t);
                        }
                    }
                    __syncthreads();
                }
            }
        }
        done += (uint64_t)hc;
        if (done >= total) break;

        // ---- exchange boundary rows with the two neighbouring stripes ----
        const int par = cyc & 1;
        uint32_t* mine = P.xbuf + ((size_t)c * 4 + (size_t)par * 2) * side_words;
        if (!bot) copy_rows_to_global(mine, srow0 + (int64_t)lo * RW, (int64_t)side_words, tid, nt);
        if (!top) copy_rows_to_global(mine + side_words, srow0 + (int64_t)(hi - h) * RW, (int64_t)side_words, tid, nt);
        __syncthreads();
        if (tid == 0) {
            const unsigned long long want = ((unsigned long long)P.epoch << 32) | (unsigned)(cyc + 1);
            __threadfence();
            st_release(P.flags + c, want);
            int ok = 1;
            const uint64_t t0 = globaltimer();
            for (int side = 0; side < 2 && ok; ++side) {
                if ((side == 0 && bot) || (side == 1 && top)) continue;
                const unsigned long long* f = P.flags + (side == 0 ? c - 1 : c + 1);
                while (ld_acquire(f) < want) {
                    if (*(volatile int*)P.status) { ok = 0; break; }
                    if (globaltimer() - t0 > kWaitLimitNs) {
                        atomicExch(P.status, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(20);
                }
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) return;   // the state is undefined; the host reports TL_ETIMEOUT
        if (!bot) {
            const uint32_t* theirs = P.xbuf + ((size_t)(c - 1) * 4 + (size_t)par * 2 + 1) * side_words;
            copy_rows_from_global(srow0 + (int64_t)(lo - h) * RW, theirs, (int64_t)side_words, tid, nt);
        }
        if (!top) {
            const uint32_t* theirs = P.xbuf + ((size_t)(c + 1) * 4 + (size_t)par * 2) * side_words;
            copy_rows_from_global(srow0 + (int64_t)hi * RW, theirs, (int64_t)side_words, tid, nt);
        }
        __syncthreads();
        ++cyc;
    }
    copy_rows_to_global(P.rows0 + (int64_t)lo * RW, srow0 + (int64_t)lo * RW, (int64_t)(hi - lo) * RW, tid, nt);
}

template <int LAT, int TK>
static const void* kernel_ptr()
{
    return reinterpret_cast<const void*>(&resident_kernel<LAT, TK>);
}

static const void* pick(int lattice, int tk)
{
    if (lattice == LAT_DOMINO) return tk == THR_SITE ? kernel_ptr<LAT_DOMINO, THR_SITE>() : kernel_ptr<LAT_DOMINO, THR_SCALAR>();
    if (lattice == LAT_LOZENGE) return tk == THR_SITE ? kernel_ptr<LAT_LOZENGE, THR_SITE>() : kernel_ptr<LAT_LOZENGE, THR_SCALAR>();
    return kernel_ptr<LAT_SIXV, THR_TABLE>();
}

int resident_prepare(const Geom& g, int thr_kind, int threads, size_t smem_bytes, int* blocks_per_sm)
{
    *blocks_per_sm = 0;
    const void* k = pick(g.lattice, thr_kind);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (int)e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem_bytes);
    if (e != cudaSuccess) cudaGetLastError();
    return (int)e;
}

int launch_resident(const Geom& g, uint32_t* rows, const ResidentPlan& plan, uint32_t sweep0,
                    uint32_t nsweeps, const DevRng& rng, const ThrView& th, const int2* grange,
                    unsigned int epoch, unsigned long long* ring, uint32_t* counts, uint64_t burn,
                    uint32_t stride, void* stream)
{
    ResParams P;
    P.rows0 = rows + g.row_words;
    P.g = g;
    P.stripe_lo = plan.stripe_lo;
    P.halo = plan.halo;
    P.sweep0 = sweep0;
    P.nsweeps = nsweeps;
    P.rng = rng;
    P.th = th;
    P.grange = grange;
    P.xbuf = plan.xbuf;
    P.flags = plan.flags;
    P.status = plan.status;
    P.ring = ring;
    P.counts = counts;
    P.burn = burn;
    P.stride = stride;
    P.epoch = epoch;
    void* args[] = {&P};
    const void* k = pick(g.lattice, th.kind);
    return (int)cudaLaunchCooperativeKernel(k, dim3(plan.ctas), dim3(plan.threads), args, plan.smem_bytes,
                                            reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace tl
