// Shared-memory resident multi-sweep kernel (cooperative launch).
//
// The paper launches Rotate and Update once per half-step and moves the
// whole tiling through device memory every time (Sec. 2.2).  Here one launch
// runs many sweeps: each CTA keeps a horizontal stripe of the packed state
// plus `halo` rows above and below it in shared memory.  A pass updates every
// row whose inputs are still exact; because a site only reads edges within
// one row of it, the exact region shrinks by one row at each interior stripe
// edge per pass, so after `halo` passes the CTA still holds its own rows
// exactly.  It then publishes its top and bottom `halo` rows and refreshes its
// halos from its two neighbours.  State crosses the memory system once per
// `halo` passes and only at stripe seams; otherwise it stays on chip.
//
// Within a cycle of `halo` passes the work is split in two phases:
//  1. random planes: the first `npre` Philox planes of every group the cycle
//     will touch are generated up front into shared memory -- independent
//     work that keeps the integer pipes busy;
//  2. passes: each active 128-site group (from a per-CTA item table that
//     lists only groups holding domain sites) reads its planes from shared
//     memory, so a pass is a short chain of shared-memory loads and bitwise
//     logic; planes beyond `npre` are generated on the spot when needed.
//
// Exchange: every boundary word travels with a 32-bit tag (launch epoch,
// cycle) in one 64-bit store; the reader polls the 64-bit words until the
// tags match, so no separate fence or flag round trip is needed.  Buffers are
// double-buffered by cycle parity.  Every wait is bounded (2 s); on expiry the
// CTA raises the status word and returns.
#include "tl_device.cuh"

#include <cstdint>

namespace tl {

struct ResParams {
    uint32_t* rows0;            // global row 0 (after the pad row)
    Geom g;
    const int* stripe_lo;
    int halo, npre;
    const uint8_t* colours;     // random pass order: colour of every slot of the launch, else nullptr
    int cap_items;              // item-table capacity per CTA
    int cap_cycle;              // random-plane buffer capacity (groups per cycle)
    uint32_t sweep0, nsweeps;
    DevRng rng;
    ThrView th;
    const int2* grange;
    unsigned long long* xbuf;   // tagged exchange words
    int* status;
    unsigned long long* ring;
    uint32_t* counts;           // bit-sliced density counter planes, or nullptr
    uint64_t burn;
    uint32_t stride;
    unsigned int epoch;
    unsigned long long* flips;  // accepted-flip counter, or nullptr
};

TL_DEV uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
TL_DEV unsigned long long ld_relaxed(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
TL_DEV void st_relaxed(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

TL_DEV void ld_relaxed2(const unsigned long long* p, unsigned long long* a, unsigned long long* b)
{
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(*a), "=l"(*b) : "l"(p) : "memory");
}
TL_DEV void st_relaxed2(unsigned long long* p, unsigned long long a, unsigned long long b)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: far beyond any healthy exchange

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

// Item range of pass i (1-based) of a cycle: table `tab` entries [s, e).
struct PassRange {
    int tab, s, e;
};

template <int LAT>
TL_DEV PassRange pass_range(const Geom& g, int i, uint32_t pass, int slo, int shi, bool bot, bool top,
                            const int* off, int nloc)
{
    const int vlo = bot ? -1 : slo + (i - 1);
    const int vhi = top ? g.H + 1 : shi - (i - 1);
    PassRange r;
    if (LAT == LAT_SIXV) {
        // face rows Y in [max(vlo,1), min(vhi-2, N-1)] of the class parity
        const int a = vlo > 1 ? vlo : 1;
        const int last = (vhi - 2) < (g.N - 1) ? (vhi - 2) : (g.N - 1);
        r.tab = sixv_py(pass);
        if (last < a) {
            r.s = r.e = 0;
            return r;
        }
        const int* o = off + r.tab * (nloc + 1);
        r.s = o[a - slo];
        r.e = o[last + 1 - slo];
    } else {
        const int a = (vlo + 1) > 0 ? (vlo + 1) : 0;
        const int b = vhi < g.H ? vhi : g.H;
        r.tab = 0;
        if (b <= a) {
            r.s = r.e = 0;
            return r;
        }
        r.s = off[a - slo];
        r.e = off[b - slo];
    }
    return r;
}

// FAST: dominoes at t = 2^31 with the branch-free, atomic-free group update;
// every updater thread handles at most two groups per pass.
template <int LAT, int TK, int NT, bool FAST>
__global__ void __launch_bounds__(NT, 1) resident_kernel(const ResParams P)
{
    extern __shared__ uint4 smem4[];
    __shared__ int s_ok;
    __shared__ unsigned long long s_red[NT / 32];
    __shared__ int4 s_ptab[64];
    __shared__ uint32_t s_psweep[64];
    __shared__ uint32_t s_next_sweep, s_next_pass;
    __shared__ __align__(16) uint32_t s_ttab[LAT == LAT_SIXV ? 32 * 16 : 4];   // expanded six-vertex table
    __shared__ __align__(16) uint32_t s_ctab[LAT == LAT_SIXV ? 32 * 8 : 4];    // expanded count table
    const Geom& g = P.g;
    const int64_t RW = g.row_words;
    const int c = blockIdx.x, C = gridDim.x;
    const int tid = threadIdx.x;
    const int lo = P.stripe_lo[c], hi = P.stripe_lo[c + 1];
    const bool bot = (c == 0), top = (c == C - 1);
    const int h = P.halo;
    const int slo = bot ? -1 : lo - h;
    const int shi = top ? g.H + 1 : hi + h;
    const int nloc = shi - slo;
    constexpr int NTAB = (LAT == LAT_SIXV) ? 2 : 1;

    // shared memory carve-up: rows | random planes | item table | offsets
    uint32_t* sm = reinterpret_cast<uint32_t*>(smem4);
    uint32_t* srow0 = sm - (int64_t)slo * RW;   // srow0 + y * RW is global row y
    uint4* rbuf = reinterpret_cast<uint4*>(sm + (int64_t)nloc * RW);
    uint32_t* items = reinterpret_cast<uint32_t*>(rbuf + (size_t)P.npre * P.cap_cycle);
    int* off = reinterpret_cast<int*>(items + P.cap_items);
    // FAST only: 8-byte aligned after the offsets
    uint2* fitems = reinterpret_cast<uint2*>((reinterpret_cast<uintptr_t>(off + NTAB * (nloc + 1)) + 7) & ~(uintptr_t)7);

    copy_rows_from_global(sm, P.rows0 + (int64_t)slo * RW, (int64_t)nloc * RW, tid, NT);
    if (LAT == LAT_SIXV) {
        for (int i = tid; i < 32 * 16; i += NT) s_ttab[i] = ((P.th.tmask[i >> 4] >> (i & 15)) & 1u) ? 0xFFFFFFFFu : 0u;
        for (int i = tid; i < 32 * 8; i += NT) {
            const int n = i & 7;
            s_ctab[i] = (n < 5 && ((P.th.t5[n] >> (31 - (i >> 3))) & 1u)) ? 0xFFFFFFFFu : 0u;
        }
    }
    const uint32_t* ctab = (LAT == LAT_SIXV && P.th.cpol >= 0) ? s_ctab : nullptr;

    // item tables: active groups of each local row (six-vertex: one table per
    // face-row parity), prefix offsets per table
    for (int t = 0; t < NTAB; ++t)
        for (int r = tid; r < nloc; r += NT) {
            const int y = slo + r;
            int cnt = 0;
            if (y >= 0 && y < g.H && (NTAB == 1 || (y & 1) == t)) {
                const int2 gr = P.grange[y];
                cnt = gr.y > gr.x ? gr.y - gr.x : 0;
            }
            off[t * (nloc + 1) + r + 1] = cnt;
        }
    __syncthreads();
    if (tid == 0) {
        // absolute offsets: the tables are stored one after the other
        int run = 0;
        for (int t = 0; t < NTAB; ++t) {
            int* o = off + t * (nloc + 1);
            o[0] = run;
            for (int r = 0; r < nloc; ++r) o[r + 1] += o[r];
            run = o[nloc];
        }
    }
    __syncthreads();
    for (int t = 0; t < NTAB; ++t)
        for (int r = tid; r < nloc; r += NT) {
            const int y = slo + r;
            if (y < 0 || y >= g.H || (NTAB == 2 && (y & 1) != t)) continue;
            const int2 gr = P.grange[y];
            int o = off[t * (nloc + 1) + r];
            for (int m = gr.x; m < gr.y; ++m) {
#ifdef TL_DEBUG
                if (!TL_IN(o, P.cap_items, 201)) break;
#endif
                if (FAST) {
                    // word offset of (row y, plane 0, word 4m) and whether m+1 follows in this row
                    fitems[o] = make_uint2((uint32_t)((int64_t)r * RW + 4 * m),
                                           (uint32_t)y | ((uint32_t)m << 16) | (m + 1 < gr.y ? 0x80000000u : 0u));
                }
                items[o++] = ((uint32_t)r << 8) | (uint32_t)m;
            }
        }
    __syncthreads();

    const int passes = g.passes;
    const uint64_t total = (uint64_t)P.nsweeps * passes;
    const size_t side_words = (size_t)h * RW;
    const int cap = P.cap_cycle;
    // warp roles: the first half updates the current pass, the second half
    // generates the random planes of the next pass
    constexpr int HALF = NT / 2;
    const bool upd_role = tid < HALF;
    const int rtid = upd_role ? tid : tid - HALF;
    uint64_t done = 0;
    int cyc = 0;
    // the next density sample: sweeps s (counted after the sweep, 1-based)
    // with s >= burn and (s - burn) % stride == 0, tracked incrementally
    uint64_t next_sample = ~0ull;
    if (P.counts && P.stride) {
        const uint64_t first = (uint64_t)P.sweep0 + 1;
        next_sample = first <= P.burn ? P.burn : P.burn + ((first - P.burn + P.stride - 1) / P.stride) * P.stride;
    }
    uint32_t nflip = 0;   // accepted flips of this thread's owned sites
    uint32_t cyc_sweep = P.sweep0, cyc_pass = 0;   // first pass of the current cycle
    // pass table of a cycle: item range, random-plane offset, pass slot |
    // colour << 8, sweep.  The slot keys the random numbers, the colour (the
    // slot itself unless the order is random) selects the sites.  Built by
    // the first generator thread.
    auto build_table = [&](int hc_, uint32_t sweep, uint32_t pass) {
        int base = 0;
        for (int i = 1; i <= hc_; ++i) {
            const uint32_t colour = P.colours ? P.colours[(size_t)(sweep - P.sweep0) * passes + pass] : pass;
            const PassRange pr = pass_range<LAT>(g, i, colour, slo, shi, bot, top, off, nloc);
            s_ptab[i - 1] = make_int4(pr.s, pr.e - pr.s, base, (int)(pass | (colour << 8)));
            s_psweep[i - 1] = sweep;
            base += pr.e - pr.s;
            if (++pass == (uint32_t)passes) {
                pass = 0;
                ++sweep;
            }
        }
        s_next_sweep = sweep;
        s_next_pass = pass;
    };
    // random planes of one pass (generator warps): per group, four planes
    // at a time -- independent Philox chains the scheduler interleaves
    // (computing all four even when fewer are kept measured faster than
    // guarding them, and than spreading single planes over threads)
    auto gen = [&](int i) {
        const int4 e = s_ptab[i];
        const uint32_t sweep = s_psweep[i], pass = (uint32_t)e.w & 255u;   // slot
        for (int it = rtid; it < e.y; it += HALF) {
#ifdef TL_DEBUG
            if (!TL_IN(e.x + it, P.cap_items, 202) || !TL_IN(e.z + it, cap, 203)) continue;
#endif
            const uint32_t item = items[e.x + it];
            const int y = slo + (int)(item >> 8), m = (int)(item & 255u);
            const uint32_t grp = (uint32_t)(((LAT == LAT_SIXV) ? (y >> 1) : y) * g.Kg + m);
            for (int k0 = 0; k0 < P.npre; k0 += 4) {
                uint4 o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    o[q] = philox10(grp, sweep, ((uint32_t)(k0 + q) << 16) | pass, P.rng.stream, P.rng.k0,
                                    P.rng.k1);
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (k0 + q < P.npre) rbuf[(size_t)(k0 + q) * cap + e.z + it] = o[q];
            }
        }
    };
    // the first cycle's table and random planes; later cycles get theirs from
    // the generator warps while the updater warps exchange boundary rows
    int hc = (int)(total < (uint64_t)h ? total : (uint64_t)h);
    if (tid == HALF) build_table(hc, cyc_sweep, cyc_pass);
    __syncthreads();
    if (!upd_role) gen(0);
    __syncthreads();
    while (true) {
        const uint32_t next_sweep = s_next_sweep, next_pass = s_next_pass;
        for (int i = 0; i < hc; ++i) {
            const int4 e = s_ptab[i];
            const uint32_t sweep = s_psweep[i], slot = (uint32_t)e.w & 255u, pass = (uint32_t)e.w >> 8;
            if (FAST && upd_role) {
                // read and decide every group of the pass, then store: groups
                // read their neighbours' boundary words
                constexpr int MAXI = NT >= 1024 ? 1 : 2;
                DominoFast r[MAXI];
                bool has[MAXI];
#pragma unroll
                for (int q = 0; q < MAXI; ++q) {
                    const int it = rtid + q * HALF;
                    has[q] = it < e.y;
#ifdef TL_DEBUG
                    if (has[q] && !(TL_IN(e.x + it, P.cap_items, 204) && TL_IN(e.z + it + 1, cap + 1, 205)))
                        has[q] = false;
#endif
                    if (!has[q]) continue;
                    // {smem word offset of (y, k0), y | m << 16 | next-adjacent << 31}
                    const uint2 fi = fitems[e.x + it];
#ifdef TL_DEBUG
                    // the update reads rows y - 1 and y of the local rows
                    if (!TL_IN((int64_t)fi.x - RW, (int64_t)(nloc - 1) * RW, 206)) {
                        has[q] = false;
                        continue;
                    }
#endif
                    const int y = (int)(fi.y & 0xFFFFu), m = (int)((fi.y >> 16) & 0xFFu);
                    const uint32_t onext = (fi.y >> 31) ? rbuf[e.z + it + 1].x : 0u;
                    r[q] = domino_fast_compute(sm + fi.x, RW, g.K, (int)((pass + (uint32_t)y) & 1u), m << 2,
                                               rbuf[e.z + it], onext);
                    if (y >= lo && y < hi) nflip += r[q].nfl;
                }
                asm volatile("bar.sync 1, %0;" ::"r"(HALF) : "memory");
#pragma unroll
                for (int q = 0; q < MAXI; ++q)
                    if (has[q]) domino_fast_store(r[q]);
            } else if (!FAST && upd_role) {
                for (int it = rtid; it < e.y; it += HALF) {
#ifdef TL_DEBUG
                    if (!TL_IN(e.x + it, P.cap_items, 207) || !TL_IN(e.z + it, cap, 203)) continue;
                    // dominoes and lozenges read rows y - 1 and y, a six-vertex
                    // face row the vertex rows y and y + 1
                    if (!TL_IN((int)(items[e.x + it] >> 8) - (LAT == LAT_SIXV ? 0 : 1), nloc - 1, 208)) continue;
#endif
                    const uint32_t item = items[e.x + it];
                    const int y = slo + (int)(item >> 8), m = (int)(item & 255u);
                    const uint32_t grp = (uint32_t)(((LAT == LAT_SIXV) ? (y >> 1) : y) * g.Kg + m);
                    const RndPre rnd{rbuf + e.z + it, P.npre, cap, RndPhilox{grp, sweep, slot, P.rng}};
                    // a six-vertex face row y touches vertex rows y and y + 1
                    // and is this stripe's if its lower row is
                    group_update<LAT, TK>(srow0 + (int64_t)y * RW, RW, g, y, m, pass, rnd, P.th,
                                          LAT == LAT_SIXV ? s_ttab : nullptr, ctab,
                                          (P.flips && y >= lo && y < hi) ? &nflip : nullptr);
                }
            } else if (i + 1 < hc) {
                gen(i + 1);
            }
            __syncthreads();
            if (slot == (uint32_t)(passes - 1)) {
                // end of a sweep: the owned rows are exact (i < halo)
                const bool sample = (uint64_t)sweep + 1 == next_sample;
                if (sample) next_sample += P.stride;
                if (P.ring || sample) {
                    const int rw = (int)RW;
                    const int nw = (hi - lo) * rw;
                    const uint32_t* rb = srow0 + (int64_t)lo * RW;
                    uint64_t acc = 0;
                    for (int w = tid; w < nw; w += NT) {
                        const uint32_t v = rb[w];
                        if (!v) continue;
                        const int rr = w / rw;
                        const int rem = w - rr * rw;
                        const int pl = rem / g.K, k = rem - pl * g.K;
                        if (P.ring) acc += word_hash(v, g, lo + rr, pl, k);
                        if (sample)
                            word_count_sliced(v, (int64_t)(lo + rr) * rw + rem, (int64_t)g.H * rw, P.counts);
                    }
                    if (P.ring) {
                        for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
                        if ((tid & 31) == 0) s_red[tid >> 5] = acc;
                        __syncthreads();
                        if (tid == 0) {
                            unsigned long long t = 0;
                            for (int wv = 0; wv < NT / 32; ++wv) t += s_red[wv];
#ifdef TL_DEBUG
                            if (TL_IN(sweep - P.sweep0, P.nsweeps, 209))
#endif
                                atomicAdd(P.ring + (sweep - P.sweep0), t);
                        }
                    }
                    __syncthreads();
                }
            }
        }
        cyc_sweep = next_sweep;
        cyc_pass = next_pass;
        done += (uint64_t)hc;
        if (done >= total) break;
        const int hc_next = (int)((total - done) < (uint64_t)h ? (total - done) : (uint64_t)h);
        int ok = 1;
        if (!upd_role) {
            // the next cycle's pass table and first random planes (they touch
            // no rows, so they overlap the exchange)
            if (tid == HALF) build_table(hc_next, cyc_sweep, cyc_pass);
            asm volatile("bar.sync 2, %0;" ::"r"(HALF) : "memory");
            gen(0);
        } else {
            // ---- exchange: tagged 64-bit words, double-buffered by cycle parity ----
            const int par = cyc & 1;
            const unsigned long long tag =
                ((unsigned long long)(((P.epoch & 0xFFFFu) << 16) | (unsigned)((cyc + 1) & 0xFFFF))) << 32;
            unsigned long long* mine = P.xbuf + ((size_t)c * 4 + (size_t)par * 2) * side_words;
            const size_t half = side_words / 2;   // 16-byte units per side (side_words is a multiple of 4)
            if (!bot) {
                const uint32_t* src = srow0 + (int64_t)lo * RW;
                for (size_t w = rtid; w < half; w += HALF) st_relaxed2(mine + 2 * w, tag | src[2 * w], tag | src[2 * w + 1]);
            }
            if (!top) {
                const uint32_t* src = srow0 + (int64_t)(hi - h) * RW;
                for (size_t w = rtid; w < half; w += HALF)
                    st_relaxed2(mine + side_words + 2 * w, tag | src[2 * w], tag | src[2 * w + 1]);
            }
            // every updater thread polls its 16-byte units of both sides with loads in flight
            constexpr int MAXU = 4;
            const uint64_t t_wait = globaltimer();
            const unsigned long long* th0 = bot ? nullptr : P.xbuf + ((size_t)(c - 1) * 4 + (size_t)par * 2 + 1) * side_words;
            const unsigned long long* th1 = top ? nullptr : P.xbuf + ((size_t)(c + 1) * 4 + (size_t)par * 2) * side_words;
            uint32_t* d0 = srow0 + (int64_t)(lo - h) * RW;
            uint32_t* d1 = srow0 + (int64_t)hi * RW;
            const int units = 2 * (int)half;   // both sides
            for (int u0 = rtid; u0 < units && ok; u0 += MAXU * HALF) {
                unsigned long long a[MAXU], b[MAXU];
                unsigned need = 0;
    #pragma unroll
                for (int q = 0; q < MAXU; ++q) {
                    const int u = u0 + q * HALF;
                    const bool side = u >= (int)half;
                    const unsigned long long* src = side ? th1 : th0;
                    if (u < units && src != nullptr) {
                        need |= 1u << q;
                        ld_relaxed2(src + 2 * (u - (side ? (int)half : 0)), &a[q], &b[q]);
                    }
                }
                while (need) {
    #pragma unroll
                    for (int q = 0; q < MAXU; ++q) {
                        if (!(need >> q & 1u)) continue;
                        if ((a[q] & 0xFFFFFFFF00000000ull) == tag && (b[q] & 0xFFFFFFFF00000000ull) == tag) {
                            const int u = u0 + q * HALF;
                            const bool side = u >= (int)half;
                            uint32_t* d = (side ? d1 : d0) + 2 * (u - (side ? (int)half : 0));
                            d[0] = (uint32_t)a[q];
                            d[1] = (uint32_t)b[q];
                            need &= ~(1u << q);
                        }
                    }
                    if (!need) break;
                    if (*(volatile int*)P.status || globaltimer() - t_wait > kWaitLimitNs) {
                        atomicExch(P.status, 1);
                        ok = 0;
                        break;
                    }
                    __nanosleep(32);
    #pragma unroll
                    for (int q = 0; q < MAXU; ++q) {
                        if (!(need >> q & 1u)) continue;
                        const int u = u0 + q * HALF;
                        const bool side = u >= (int)half;
                        ld_relaxed2((side ? th1 : th0) + 2 * (u - (side ? (int)half : 0)), &a[q], &b[q]);
                    }
                }
            }
        }
        // a status word raised anywhere (a wait that gave up in another CTA,
        // or raised by the host) ends every CTA at its next exchange
        if (tid == 0) s_ok = *(volatile int*)P.status ? 0 : 1;
        __syncthreads();
        if (!ok) s_ok = 0;
        __syncthreads();
        if (!s_ok) return;   // the state is undefined; the host reports TL_ETIMEOUT
        hc = hc_next;
        ++cyc;
    }
    copy_rows_to_global(P.rows0 + (int64_t)lo * RW, srow0 + (int64_t)lo * RW, (int64_t)(hi - lo) * RW, tid, NT);
    if (P.flips && nflip) atomicAdd(P.flips, (unsigned long long)nflip);
}

template <int LAT, int TK>
static const void* kernel_ptr(int threads)
{
    return threads > 512 ? reinterpret_cast<const void*>(&resident_kernel<LAT, TK, 1024, false>)
                         : reinterpret_cast<const void*>(&resident_kernel<LAT, TK, 512, false>);
}

static const void* pick(int lattice, int tk, int threads, bool fast = false)
{
    if (fast)
        return threads > 512 ? reinterpret_cast<const void*>(&resident_kernel<LAT_DOMINO, THR_SCALAR, 1024, true>)
                             : reinterpret_cast<const void*>(&resident_kernel<LAT_DOMINO, THR_SCALAR, 512, true>);
    if (lattice == LAT_DOMINO)
        return tk == THR_SITE ? kernel_ptr<LAT_DOMINO, THR_SITE>(threads) : kernel_ptr<LAT_DOMINO, THR_SCALAR>(threads);
    if (lattice == LAT_LOZENGE)
        return tk == THR_SITE ? kernel_ptr<LAT_LOZENGE, THR_SITE>(threads) : kernel_ptr<LAT_LOZENGE, THR_SCALAR>(threads);
    return kernel_ptr<LAT_SIXV, THR_TABLE>(threads);
}

int resident_prepare(const Geom& g, int thr_kind, int threads, bool fast, size_t smem_bytes, int* blocks_per_sm)
{
    *blocks_per_sm = 0;
    const void* k = pick(g.lattice, thr_kind, threads, fast);
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
                    uint32_t stride, const uint8_t* colours, unsigned long long* flips, void* stream)
{
    ResParams P;
    P.flips = flips;
    P.rows0 = rows + g.row_words;
    P.g = g;
    P.stripe_lo = plan.stripe_lo;
    P.halo = plan.halo;
    P.npre = plan.npre;
    P.colours = colours;
    P.cap_items = plan.cap_items;
    P.cap_cycle = plan.cap_cycle;
    P.sweep0 = sweep0;
    P.nsweeps = nsweeps;
    P.rng = rng;
    P.th = th;
    P.grange = grange;
    P.xbuf = plan.xbuf;
    P.status = plan.status;
    P.ring = ring;
    P.counts = counts;
    P.burn = burn;
    P.stride = stride;
    P.epoch = epoch;
    void* args[] = {&P};
    const void* k = pick(g.lattice, th.kind, plan.threads, plan.fast);
    return (int)cudaLaunchCooperativeKernel(k, dim3(plan.ctas), dim3(plan.threads), args, plan.smem_bytes,
                                            reinterpret_cast<cudaStream_t>(stream));
}

// Colours of the pass slots of sweeps sweep0 .. sweep0 + nsweeps - 1 under
// the random pass order: out[s * passes + i] for slot i of sweep sweep0 + s.
__global__ void slot_colours_kernel(uint8_t* __restrict__ out, uint32_t sweep0, uint32_t nsweeps, int passes,
                                    DevRng rng)
{
    const uint64_t n = (uint64_t)nsweeps * passes;
    for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x)
        out[j] = (uint8_t)slot_colour(rng, sweep0 + (uint32_t)(j / passes), (uint32_t)(j % passes), passes);
}

int launch_slot_colours(uint8_t* out, uint32_t sweep0, uint32_t nsweeps, int passes, const DevRng& rng, void* stream)
{
    const uint64_t n = (uint64_t)nsweeps * passes;
    const uint64_t blocks = (n + 255) / 256;
    slot_colours_kernel<<<(unsigned)(blocks < 1024 ? (blocks ? blocks : 1) : 1024), 256, 0,
                          reinterpret_cast<cudaStream_t>(stream)>>>(out, sweep0, nsweeps, passes, rng);
    return (int)cudaGetLastError();
}

// This file's debug word (failures, then the id, index and bound of the
// first failed check); cudaErrorNotSupported in the normal build.
int dbg_fetch_resident(unsigned long long* out, bool clear)
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
