// Register-resident multi-sweep kernel for domino tilings at t = 2^31
// (cooperative launch, one CTA per SM).
//
// The paper moves the whole tiling through device memory twice per
// half-step (Rotate, then Update; Sec. 2.2).  Here every thread owns one
// 128-site group of two consecutive vertex rows -- 32 state words (edges Hz
// and Vt of both x parities, four words each per row) plus a copy of the Vt
// words of the row below -- and keeps them in registers for the whole
// launch.  A pass updates every site of one colour class (x + y mod 2,
// Sec. 1.1.3): each row of the pair has one parity per pass, so the update
// is straight-line bit logic on registers; the heat-bath decision at
// t = 2^31 needs only the first random plane of Philox4x32-10 (bit 31 of
// u < 2^31 iff that bit is 0).
//
// A site reads the four edges around it.  Two of them can belong to another
// thread: the W edge of a group's first site (top bit of the neighbouring
// group's odd-Hz word) and the Vt edges shared with the row pairs above and
// below.  After the pass every thread publishes what it flipped that others
// hold (its rows' flip masks, and the two boundary bits), one CTA barrier
// later every thread applies its neighbours' flips.  One barrier per pass;
// shared memory carries 36 bytes per thread and pass.
//
// Between CTAs the stripes exchange boundary rows every `halo` passes (the
// halo rows are recomputed redundantly, the exact region shrinking by one
// row per pass; rows whose results can no longer reach the owned stripe are
// skipped).  Boundary rows travel packed in 64-bit words of 61 data bits
// and a 3-bit cycle tag, double buffered by cycle parity (the buffers are
// cleared before every launch); every wait is bounded (2 s) and raises a
// status word instead of hanging.
#include "tl_device.cuh"

#include <cstdint>
#include <type_traits>

namespace tl {

struct RegParams {
    uint32_t* rows0;            // global row 0 (after the pad row)
    Geom g;
    const int* stripe_lo;       // [C + 1] even row bounds
    const int2* hull;           // [pairs] groups [x, y) held for rows (2q, 2q + 1)
    int halo;                   // rows per side = passes per exchange cycle (even)
    const uint8_t* colours;     // random pass order: colour of every slot, else nullptr
    uint32_t sweep0, nsweeps;
    DevRng rng;
    unsigned long long* xbuf;   // [C][2][2][halo / 2][16][Kg][2] tagged words
    int* status;
    unsigned long long* ring;
    uint32_t* counts;
    uint64_t burn;
    uint32_t stride;
    unsigned int epoch;
    unsigned long long* flips;  // accepted-flip counter, or nullptr
};

TL_DEV uint64_t rd_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
TL_DEV void rd_ld2(const unsigned long long* p, unsigned long long* a, unsigned long long* b)
{
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(*a), "=l"(*b) : "l"(p) : "memory");
}
TL_DEV void rd_st2(unsigned long long* p, unsigned long long a, unsigned long long b)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}

constexpr uint64_t kRegWaitLimitNs = 2000000000ull;   // 2 s: far beyond any healthy exchange

// One row at parity 0 (sites x = 2j): E = Hz(2j) (even plane), W = Hz(2j-1)
// (odd plane shifted up by one site; bit 0 from `pv`, the top bit of the
// left group's odd word), N = Vt(2j, y), S = Vt(2j, y-1).  Returns the flip
// mask and applies it to the row's own words; `lb` receives bit 0 of the
// mask (the flip of the left group's odd-Hz top bit).
TL_DEV uint4 row_par0(uint4& He, uint4& Ho, uint32_t& pv, uint4& N, uint4& S, uint4 o, uint32_t& lb)
{
    const uint4 Wd = shl1(Ho, pv);
    uint4 fl;
#define TL_RG_F(c)                                                                                  \
    {                                                                                               \
        const uint32_t f = (He.c & Wd.c & ~(N.c | S.c)) | (N.c & S.c & ~(He.c | Wd.c));           \
        fl.c = f & (~o.c ^ He.c);                                                                   \
    }
    TL_RG_F(x) TL_RG_F(y) TL_RG_F(z) TL_RG_F(w)
#undef TL_RG_F
    He = x4(He, fl);
    N = x4(N, fl);
    S = x4(S, fl);
    Ho.x ^= (fl.x >> 1) | (fl.y << 31);
    Ho.y ^= (fl.y >> 1) | (fl.z << 31);
    Ho.z ^= (fl.z >> 1) | (fl.w << 31);
    Ho.w ^= fl.w >> 1;
    pv ^= fl.x << 31;
    lb = fl.x & 1u;
    return fl;
}

// One row at parity 1 (sites x = 2j + 1): E = Hz(2j+1) (odd plane), W =
// Hz(2j) (even plane), N = Vt(2j+1, y), S = Vt(2j+1, y-1).  `rb` receives the
// top bit of the mask (the last site's E edge is the right group's `pv`).
TL_DEV uint4 row_par1(uint4& He, uint4& Ho, uint4& N, uint4& S, uint4 o, uint32_t& rb)
{
    uint4 fl;
#define TL_RG_F(c)                                                                                  \
    {                                                                                               \
        const uint32_t f = (Ho.c & He.c & ~(N.c | S.c)) | (N.c & S.c & ~(Ho.c | He.c));           \
        fl.c = f & (~o.c ^ Ho.c);                                                                   \
    }
    TL_RG_F(x) TL_RG_F(y) TL_RG_F(z) TL_RG_F(w)
#undef TL_RG_F
    He = x4(He, fl);
    Ho = x4(Ho, fl);
    N = x4(N, fl);
    S = x4(S, fl);
    rb = fl.w >> 31;
    return fl;
}

// The 32 words of a pair as the exchange sends them: row y0 then row y0 + 1,
// each He, Ho, Ve, Vo.
struct PairWords {
    uint4 v[8];
};

// Exchange format: the pair's 1,024 state bits (the 32 words above, word j
// holding stream bits [32j, 32j + 32)) in 17 fields of 61 bits, each field
// in the low bits of a 64-bit word whose top 3 bits carry the cycle tag;
// field 17 carries the tag alone.  Nine 16-byte units per pair and group
// instead of sixteen 32-bit words each with a 32-bit tag.  A 64-bit access
// is single-copy atomic, so a field whose tag is current holds current data.
constexpr int kXFields = 18, kXUnits = 9;
constexpr unsigned long long kXMask = (1ull << 61) - 1;

TL_DEV unsigned long long pack61(const uint32_t (&w)[32], int i)
{
    const int lo = 61 * i;
    if (lo >= 1024) return 0ull;
    const int wi = lo >> 5, s = lo & 31;
    unsigned long long x = (unsigned long long)w[wi] >> s;
    if (wi + 1 < 32) x |= (unsigned long long)w[wi + 1] << (32 - s);
    if (s > 3 && wi + 2 < 32) x |= (unsigned long long)w[wi + 2] << (64 - s);
    return x & kXMask;
}

// word j of the stream from fields with their tags cleared
TL_DEV uint32_t unpack61(const unsigned long long (&f)[kXFields], int j)
{
    const int lo = 32 * j, i0 = lo / 61, o = lo - 61 * i0;
    unsigned long long x = f[i0] >> o;
    if (61 - o < 32) x |= f[i0 + 1] << (61 - o);
    return (uint32_t)x;
}

// A density sample of one row pair: its eight 4-word blocks (rows y0 and
// y0 + 1, planes He, Ho, Ve, Vo; block j at counter word i0 + (j / 4) RW +
// (j % 4) K) are added to the bit-sliced counters together, counter plane
// by counter plane.  All reads of a plane are issued before any write, so a
// sample is one chain of dependent counter accesses, as long as the longest
// carry, instead of one chain per block.  J blocks from j0 at a time: all
// eight, or (the 512-thread build, short of registers) one row's four.
template <int J>
TL_DEV void pair_count_sliced(const PairWords& pw, int j0, int64_t i0, int64_t RW, int K, int64_t plane_words,
                              uint32_t* cplanes)
{
#ifdef TL_DEBUG
    if (!TL_IN(i0 + ((j0 + J - 1) >> 2) * RW + 3 * (int64_t)K + 3, plane_words, 107)) return;
#endif
    uint4 carry[J];
#pragma unroll
    for (int j = 0; j < J; ++j) carry[j] = pw.v[j0 + j];
    for (int b = 0; b < 32; ++b) {
        bool any = false;
#pragma unroll
        for (int j = 0; j < J; ++j) any |= any4(carry[j]);
        if (!any) break;
        uint32_t* const base = cplanes + (int64_t)b * plane_words + i0;
        uint4 c[J];
#pragma unroll
        for (int j = 0; j < J; ++j)
            c[j] = any4(carry[j]) ? *reinterpret_cast<const uint4*>(base + ((j0 + j) >> 2) * RW + ((j0 + j) & 3) * K)
                                  : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int j = 0; j < J; ++j)
            if (any4(carry[j])) {
                *reinterpret_cast<uint4*>(base + ((j0 + j) >> 2) * RW + ((j0 + j) & 3) * K) = x4(c[j], carry[j]);
                carry[j] = make_uint4(carry[j].x & c[j].x, carry[j].y & c[j].y, carry[j].z & c[j].z,
                                      carry[j].w & c[j].w);
            }
    }
}

// COUNT: the chain counts its accepted flips (a separate instantiation, so
// the default path carries no counter).  RND: the colour of every pass slot
// comes from the host's table (random order) instead of slot s updating
// colour s.
template <int NT, bool COUNT, bool RND>
__global__ void __launch_bounds__(NT, 1) regdom_kernel(const RegParams P)
{
    extern __shared__ uint4 rsm[];
    __shared__ unsigned long long s_red[NT / 32];
    const int nt = blockDim.x;
    uint4* FL0 = rsm;                                        // [2][nt] flips of row y0 (for the pair below)
    uint4* FL1 = FL0 + 2 * nt;                               // [2][nt] flips of row y0+1 (for the pair above)
    uint4* RV = FL1 + 2 * nt;                                // [nt][2] Vt words of row y0+1 (refresh)
    uint2* RH = reinterpret_cast<uint2*>(RV + 2 * nt);       // [nt] odd-Hz top words (refresh)
    uint32_t* HB = reinterpret_cast<uint32_t*>(RH + nt);     // [2][nt] boundary flip bits
    int* s_off = reinterpret_cast<int*>(HB + 2 * nt);        // [npl + 1] item offsets of the local pairs
    const Geom& g = P.g;
    const int K = g.K, Kg = g.Kg;
    const int64_t RW = g.row_words;
    const int c = blockIdx.x, C = gridDim.x, tid = threadIdx.x;
    const int lo = P.stripe_lo[c], hi = P.stripe_lo[c + 1];
    const bool bot = (c == 0), top = (c == C - 1);
    const int h = P.halo;
    const int slo = bot ? lo : lo - h;
    const int shi = top ? hi : hi + h;
    const int q0 = slo >> 1, npl = (shi - slo) >> 1;
    int2* s_hull = reinterpret_cast<int2*>((reinterpret_cast<uintptr_t>(s_off + npl + 1) + 7) & ~(uintptr_t)7);

    for (int i = tid; i < npl; i += nt) s_hull[i] = P.hull[q0 + i];
    __syncthreads();
    if (tid == 0) {
        int run = 0;
        for (int i = 0; i < npl; ++i) {
            s_off[i] = run;
            const int2 hh = s_hull[i];
            run += hh.y > hh.x ? hh.y - hh.x : 0;
        }
        s_off[npl] = run;
    }
    __syncthreads();
    const int nitems = s_off[npl];
    const bool act = tid < nitems;

    // ---- my item: pair index, group, neighbours, role ----
    int pi = 0, m = 0, ib = -1, ia = -1, il = -1, ir = -1;
    if (act) {
        int a = 0, b = npl - 1;
        while (a < b) {   // last pair whose first item is <= tid
            const int mid = (a + b + 1) >> 1;
            if (s_off[mid] <= tid) a = mid;
            else b = mid - 1;
        }
        pi = a;
        const int2 hh = s_hull[pi];
        m = hh.x + (tid - s_off[pi]);
        if (m > hh.x) il = tid - 1;
        if (m + 1 < hh.y) ir = tid + 1;
        if (pi > 0) {
            const int2 hb = s_hull[pi - 1];
            if (m >= hb.x && m < hb.y) ib = s_off[pi - 1] + (m - hb.x);
        }
        if (pi + 1 < npl) {
            const int2 ha = s_hull[pi + 1];
            if (m >= ha.x && m < ha.y) ia = s_off[pi + 1] + (m - ha.x);
        }
#ifdef TL_DEBUG
        if (ib >= 0 && !TL_IN(ib, nt, 101)) ib = -1;
        if (ia >= 0 && !TL_IN(ia, nt, 102)) ia = -1;
        if (il >= 0 && !TL_IN(il, nt, 103)) il = -1;
        if (ir >= 0 && !TL_IN(ir, nt, 104)) ir = -1;
#endif
    }
    const int y0 = slo + 2 * pi;
    const bool owned = act && y0 >= lo && y0 < hi;
    // Halo pairs are updated in pass i of a cycle while dist + i <= halo.  A
    // row's flips change its own edges and the Vt edges of the row below, so
    // a row at distance e from the stripe is needed after pass i while
    // e + i <= halo (below the stripe: dist = e of the pair's upper row,
    // 1, 3, 5, ...), and above the stripe its flips are also needed while
    // the row below it is (dist = e - 1 of the pair's lower row, 0, 2, ...).
    const int dist = owned ? 0 : (y0 < lo ? lo - (y0 + 1) : y0 - hi);

    // ---- load the state ----
    uint4 He0 = {}, Ho0 = {}, Ve0 = {}, Vo0 = {}, He1 = {}, Ho1 = {}, Ve1 = {}, Vo1 = {}, Se = {}, So = {};
    uint32_t pv0 = 0, pv1 = 0;
    const int k0 = 4 * m;
    // rows y0 - 1 .. y0 + 1 of the padded buffer (rows -1 .. H) and words
    // k0 .. k0 + 3 of a plane row
#ifdef TL_DEBUG
    const bool inb = TL_IN(y0 + 1, g.H + 1, 105) && TL_IN(k0 + 3, K, 106);
#else
    constexpr bool inb = true;
#endif
    if (act && inb) {
        const uint32_t* b0 = P.rows0 + (int64_t)y0 * RW + k0;
        const uint32_t* b1 = b0 + RW;
        const uint32_t* bs = b0 - RW;
        He0 = __ldcg(reinterpret_cast<const uint4*>(b0));
        Ho0 = __ldcg(reinterpret_cast<const uint4*>(b0 + K));
        Ve0 = __ldcg(reinterpret_cast<const uint4*>(b0 + 2 * K));
        Vo0 = __ldcg(reinterpret_cast<const uint4*>(b0 + 3 * K));
        He1 = __ldcg(reinterpret_cast<const uint4*>(b1));
        Ho1 = __ldcg(reinterpret_cast<const uint4*>(b1 + K));
        Ve1 = __ldcg(reinterpret_cast<const uint4*>(b1 + 2 * K));
        Vo1 = __ldcg(reinterpret_cast<const uint4*>(b1 + 3 * K));
        Se = __ldcg(reinterpret_cast<const uint4*>(bs + 2 * K));
        So = __ldcg(reinterpret_cast<const uint4*>(bs + 3 * K));
        if (m > 0) {
            pv0 = __ldcg(b0 + K - 1);
            pv1 = __ldcg(b1 + K - 1);
        }
    }
    const uint32_t grp0 = (uint32_t)y0 * (uint32_t)Kg + (uint32_t)m;
    const uint32_t grp1 = grp0 + (uint32_t)Kg;

    const uint64_t total = (uint64_t)P.nsweeps * 2;
    const size_t side_words = (size_t)(h >> 1) * 32 * Kg;   // u64 per side
    uint64_t done = 0;
    uint32_t nflip = 0;   // accepted flips of this thread's owned sites
    int cyc = 0;
    // the next density sample: sweeps s (counted after the sweep, 1-based)
    // with s >= burn and (s - burn) % stride == 0, tracked incrementally
    uint64_t next_sample = ~0ull;
    if (P.counts && P.stride) {
        const uint64_t first = (uint64_t)P.sweep0 + 1;
        next_sample = first <= P.burn ? P.burn : P.burn + ((first - P.burn + P.stride - 1) / P.stride) * P.stride;
    }
    uint32_t sweep = P.sweep0;
    // Random words, ping-pong by pass slot: the words of slot s are in
    // oS0 / oS1 (rows y0, y0 + 1).  A pass draws the next pass's words in
    // the same block as its own update (independent chains, interleaved);
    // they depend on no state.  Every exchange cycle has an even number of
    // passes, so cycles (and launches) start at slot 0 and the shared-memory
    // buffer of a pass is its slot.
    uint4 oA0 = {}, oA1 = {}, oB0 = {}, oB1 = {};
    if (act) {
        oA0 = philox10(grp0, sweep, 0u, P.rng.stream, P.rng.k0, P.rng.k1);
        oA1 = philox10(grp1, sweep, 0u, P.rng.stream, P.rng.k0, P.rng.k1);
    }
    // One pass: colour parity PAR1 (the parity of row y0, y0 even), slot SL.
    auto pass = [&](auto par1c, auto slc, int ip, const uint4& oc0, const uint4& oc1, uint4& on0, uint4& on1) {
        constexpr bool par1 = decltype(par1c)::value;
        constexpr int sl = decltype(slc)::value;
        const bool live = act && (dist + ip <= h);
        const uint32_t nslot = sl ^ 1, nsweep = sl ? sweep + 1 : sweep;
        uint4* const fl0 = FL0 + sl * nt;
        uint4* const fl1 = FL1 + sl * nt;
        uint32_t* const hb = HB + sl * nt;
        if (live) {
            uint4 f0, f1;
            uint32_t b0, b1;
            on0 = philox10(grp0, nsweep, nslot, P.rng.stream, P.rng.k0, P.rng.k1);
            on1 = philox10(grp1, nsweep, nslot, P.rng.stream, P.rng.k0, P.rng.k1);
            if (!par1) {
                f0 = row_par0(He0, Ho0, pv0, Ve0, Se, oc0, b0);
                f1 = row_par1(He1, Ho1, Vo1, Vo0, oc1, b1);
            } else {
                f0 = row_par1(He0, Ho0, Vo0, So, oc0, b0);
                f1 = row_par0(He1, Ho1, pv1, Ve1, Ve0, oc1, b1);
            }
            fl0[tid] = f0;
            fl1[tid] = f1;
            hb[tid] = b0 | (b1 << 1);
            if (COUNT && owned) nflip += popc4(f0) + popc4(f1);
        }
        __syncthreads();
        if (live) {
            // the pair below flipped its upper row (Vt row y0-1 at the
            // other parity); the pair above its lower row (Vt row y0+1 at
            // this parity); left / right groups their boundary bits
            const uint4 zb = make_uint4(0u, 0u, 0u, 0u);
            const uint4 fb = ib >= 0 ? fl1[ib] : zb;
            const uint4 fa = ia >= 0 ? fl0[ia] : zb;
            const uint32_t hl = il >= 0 ? hb[il] : 0u;
            const uint32_t hr = ir >= 0 ? hb[ir] : 0u;
            if (!par1) {
                So = x4(So, fb);
                Ve1 = x4(Ve1, fa);
                Ho0.w ^= (hr & 1u) << 31;          // right group's first site, row y0
                pv1 ^= ((hl >> 1) & 1u) << 31;     // left group's last site, row y0+1
            } else {
                Se = x4(Se, fb);
                Vo1 = x4(Vo1, fa);
                pv0 ^= (hl & 1u) << 31;            // left group's last site, row y0
                Ho1.w ^= ((hr >> 1) & 1u) << 31;   // right group's first site, row y0+1
            }
        }
        if constexpr (sl == 1) {
            // end of a sweep: owned rows are exact
            const bool sample = (uint64_t)sweep + 1 == next_sample;
            if (sample) next_sample += P.stride;
            if (P.ring || sample) {
                uint64_t acc = 0;
                if (owned) {
                    const PairWords pw{{He0, Ho0, Ve0, Vo0, He1, Ho1, Ve1, Vo1}};
                    if (sample) {
                        const int64_t i0 = (int64_t)y0 * RW + k0, pw_ = (int64_t)g.H * RW;
                        if (NT < 512 && y0 + 1 < g.H) {
                            pair_count_sliced<8>(pw, 0, i0, RW, K, pw_, P.counts);
                        } else {
                            pair_count_sliced<4>(pw, 0, i0, RW, K, pw_, P.counts);
                            if (y0 + 1 < g.H) pair_count_sliced<4>(pw, 4, i0, RW, K, pw_, P.counts);
                        }
                    }
                    if (P.ring) {
#pragma unroll
                        for (int r = 0; r < 2; ++r) {
                            const int y = y0 + r;
                            if (y >= g.H) continue;
#pragma unroll
                            for (int pl = 0; pl < 4; ++pl) {
                                const uint4 v4 = pw.v[4 * r + pl];
                                const uint32_t vv[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                                for (int w = 0; w < 4; ++w)
                                    if (vv[w]) acc += word_hash(vv[w], g, y, pl, k0 + w);
                            }
                        }
                    }
                }
                if (P.ring) {
                    for (int o = 16; o; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
                    if ((tid & 31) == 0) s_red[tid >> 5] = acc;
                    __syncthreads();
                    if (tid == 0) {
                        unsigned long long t = 0;
                        for (int wv = 0; wv < (nt + 31) / 32; ++wv) t += s_red[wv];
#ifdef TL_DEBUG
                        if (TL_IN(sweep - P.sweep0, P.nsweeps, 110))
#endif
                            atomicAdd(P.ring + (sweep - P.sweep0), t);
                    }
                }
            }
            sweep = nsweep;
        }
    };
    using F = std::integral_constant<bool, false>;
    using Tr = std::integral_constant<bool, true>;
    using S0 = std::integral_constant<int, 0>;
    using S1 = std::integral_constant<int, 1>;
    while (true) {
        const int hc = (int)((total - done) < (uint64_t)h ? (total - done) : (uint64_t)h);
        for (int ip = 1; ip <= hc; ip += 2) {
            if constexpr (!RND) {
                // fixed order: slot s updates colour s
                pass(F{}, S0{}, ip, oA0, oA1, oB0, oB1);
                pass(Tr{}, S1{}, ip + 1, oB0, oB1, oA0, oA1);
            } else {
                // random order: the colour of each slot from the host's table
                const uint8_t* cs = P.colours + (size_t)(sweep - P.sweep0) * 2;
                const bool p0 = (cs[0] & 1u) != 0, p1 = (cs[1] & 1u) != 0;
                if (p0) pass(Tr{}, S0{}, ip, oA0, oA1, oB0, oB1);
                else pass(F{}, S0{}, ip, oA0, oA1, oB0, oB1);
                if (p1) pass(Tr{}, S1{}, ip + 1, oB0, oB1, oA0, oA1);
                else pass(F{}, S1{}, ip + 1, oB0, oB1, oA0, oA1);
            }
        }
        done += (uint64_t)hc;
        if (done >= total) break;

        // ---- exchange of boundary rows with the neighbouring stripes ----
        const int par = cyc & 1;
        // the buffer of a cycle parity holds the data of cycle cyc - 2, or
        // zeros (cleared before every launch): a tag of cyc mod 4, plus one,
        // tells them apart
        const unsigned long long tag = (unsigned long long)((cyc & 3) + 1) << 61;
        if (owned) {
            uint32_t w[32];
            {
                const PairWords pw{{He0, Ho0, Ve0, Vo0, He1, Ho1, Ve1, Vo1}};
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    w[4 * v] = pw.v[v].x;
                    w[4 * v + 1] = pw.v[v].y;
                    w[4 * v + 2] = pw.v[v].z;
                    w[4 * v + 3] = pw.v[v].w;
                }
            }
            for (int s = 0; s < 2; ++s) {
                const bool pub = s == 0 ? (!bot && y0 < lo + h) : (!top && y0 >= hi - h);
                if (!pub) continue;
                const int idx = s == 0 ? (y0 - lo) >> 1 : (y0 - (hi - h)) >> 1;
#ifdef TL_DEBUG
                if (!TL_IN(((size_t)(c * 2 + par) * 2 + s) * side_words + (size_t)idx * 32 * Kg +
                               ((size_t)(kXUnits - 1) * Kg + m) * 2 + 1,
                           (size_t)C * 4 * side_words, 108))
                    continue;
#endif
                unsigned long long* dst = P.xbuf + ((size_t)(c * 2 + par) * 2 + s) * side_words +
                                          (size_t)idx * 32 * Kg;
#pragma unroll
                for (int u = 0; u < kXUnits; ++u)   // 16-byte unit u: fields 2u, 2u + 1
                    rd_st2(dst + ((size_t)u * Kg + m) * 2, tag | pack61(w, 2 * u), tag | pack61(w, 2 * u + 1));
            }
        }
        int ok = 1;
        if (act && !owned) {
            // halo pair: poll the neighbour's published words (both rows at
            // once); the random words of the next pass, which halo items
            // skipped at the end of the cycle, are drawn while the first
            // loads are in flight
            const bool below = y0 < lo;
            const int idx = below ? (y0 - (lo - h)) >> 1 : (y0 - hi) >> 1;
            const unsigned long long* src = P.xbuf +
                                            ((size_t)((below ? c - 1 : c + 1) * 2 + par) * 2 + (below ? 1 : 0)) *
                                                side_words +
                                            (size_t)idx * 32 * Kg;
            unsigned long long f[kXFields];
#ifdef TL_DEBUG
            if (!TL_IN(((size_t)((below ? c - 1 : c + 1) * 2 + par) * 2 + (below ? 1 : 0)) * side_words +
                           (size_t)idx * 32 * Kg + ((size_t)(kXUnits - 1) * Kg + m) * 2 + 1,
                       (size_t)C * 4 * side_words, 109)) {
                atomicExch(P.status, 1);   // reported as a failed wait; nothing is read
                ok = 0;
            }
#pragma unroll
            for (int q = 0; q < kXFields; ++q) f[q] = 0ull;
            if (ok)
#endif
#pragma unroll
                for (int q = 0; q < kXUnits; ++q) rd_ld2(src + ((size_t)q * Kg + m) * 2, &f[2 * q], &f[2 * q + 1]);
            oA0 = philox10(grp0, sweep, 0u, P.rng.stream, P.rng.k0, P.rng.k1);
            oA1 = philox10(grp1, sweep, 0u, P.rng.stream, P.rng.k0, P.rng.k1);
            const uint64_t t_wait = rd_globaltimer();
            unsigned need = (1u << kXUnits) - 1;
            while (true) {
#pragma unroll
                for (int q = 0; q < kXUnits; ++q)
                    if ((need >> q & 1u) && (f[2 * q] & ~kXMask) == tag && (f[2 * q + 1] & ~kXMask) == tag)
                        need &= ~(1u << q);
                if (!need) break;
                if (*(volatile int*)P.status || rd_globaltimer() - t_wait > kRegWaitLimitNs) {
                    atomicExch(P.status, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
#pragma unroll
                for (int q = 0; q < kXUnits; ++q)
                    if (need >> q & 1u) rd_ld2(src + ((size_t)q * Kg + m) * 2, &f[2 * q], &f[2 * q + 1]);
            }
            if (ok) {
#pragma unroll
                for (int q = 0; q < kXFields; ++q) f[q] &= kXMask;
#define TL_RG_W(v) make_uint4(unpack61(f, 4 * (v)), unpack61(f, 4 * (v) + 1), unpack61(f, 4 * (v) + 2), unpack61(f, 4 * (v) + 3))
                He0 = TL_RG_W(0); Ho0 = TL_RG_W(1); Ve0 = TL_RG_W(2); Vo0 = TL_RG_W(3);
                He1 = TL_RG_W(4); Ho1 = TL_RG_W(5); Ve1 = TL_RG_W(6); Vo1 = TL_RG_W(7);
#undef TL_RG_W
            }
        }
        // copies of the row below (Vt) and of the left group's odd-Hz top
        // words from the neighbouring items, now exact again
        if (act) {
            RV[2 * tid] = Ve1;
            RV[2 * tid + 1] = Vo1;
            RH[tid] = make_uint2(Ho0.w, Ho1.w);
        }
        // a status word raised anywhere (a wait that gave up in another CTA,
        // or raised by the host) ends every CTA at its next exchange
        if (tid == 0 && *(volatile int*)P.status) ok = 0;
        if (!__syncthreads_and(ok)) return;   // the state is undefined; the host reports TL_ETIMEOUT
        if (act) {
            if (ib >= 0) {
                Se = RV[2 * ib];
                So = RV[2 * ib + 1];
            }
            if (il >= 0) {
                const uint2 r = RH[il];
                pv0 = r.x;
                pv1 = r.y;
            }
        }
        ++cyc;
    }
    if (COUNT && nflip) atomicAdd(P.flips, (unsigned long long)nflip);
    if (owned && inb) {
        uint32_t* b0 = P.rows0 + (int64_t)y0 * RW + k0;
        __stcg(reinterpret_cast<uint4*>(b0), He0);
        __stcg(reinterpret_cast<uint4*>(b0 + K), Ho0);
        __stcg(reinterpret_cast<uint4*>(b0 + 2 * K), Ve0);
        __stcg(reinterpret_cast<uint4*>(b0 + 3 * K), Vo0);
        if (y0 + 1 < g.H) {
            uint32_t* b1 = b0 + RW;
            __stcg(reinterpret_cast<uint4*>(b1), He1);
            __stcg(reinterpret_cast<uint4*>(b1 + K), Ho1);
            __stcg(reinterpret_cast<uint4*>(b1 + 2 * K), Ve1);
            __stcg(reinterpret_cast<uint4*>(b1 + 3 * K), Vo1);
        }
    }
}

template <bool COUNT, bool RND>
static const void* reg_pick_nt(int threads)
{
    if (threads > 384) return reinterpret_cast<const void*>(&regdom_kernel<512, COUNT, RND>);
    if (threads > 256) return reinterpret_cast<const void*>(&regdom_kernel<384, COUNT, RND>);
    return reinterpret_cast<const void*>(&regdom_kernel<256, COUNT, RND>);
}

static const void* reg_pick(int threads, bool count, bool rnd)
{
    if (count) return rnd ? reg_pick_nt<true, true>(threads) : reg_pick_nt<true, false>(threads);
    return rnd ? reg_pick_nt<false, true>(threads) : reg_pick_nt<false, false>(threads);
}

size_t regdom_smem_bytes(int threads, int max_local_pairs)
{
    // FL0, FL1: 2 x 2 x threads uint4; RV: 2 x threads uint4; RH: threads
    // uint2; HB: 2 x threads u32; offsets (pairs + 2) ints; hulls (pairs) int2
    size_t b = (size_t)threads * (16 * 6 + 8 + 8);
    b += (size_t)(max_local_pairs + 2) * 4;
    b = (b + 7) & ~(size_t)7;
    b += (size_t)max_local_pairs * 8;
    return b;
}

int regdom_prepare(int threads, size_t smem_bytes, int* blocks_per_sm)
{
    *blocks_per_sm = 0;
    const void* k = reg_pick(threads, false, false);
    cudaError_t e = cudaSuccess;
    for (int v = 0; v < 4 && e == cudaSuccess; ++v)
        e = cudaFuncSetAttribute(reg_pick(threads, (v & 1) != 0, (v & 2) != 0),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return (int)e;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, threads, smem_bytes);
    if (e != cudaSuccess) cudaGetLastError();
    return (int)e;
}

int launch_regdom(const Geom& g, uint32_t* rows, const RegPlan& plan, uint32_t sweep0, uint32_t nsweeps,
                  const DevRng& rng, unsigned int epoch, unsigned long long* ring, uint32_t* counts, uint64_t burn,
                  uint32_t stride, const uint8_t* colours, unsigned long long* flips, void* stream)
{
    RegParams P;
    P.flips = flips;
    P.rows0 = rows + g.row_words;
    P.g = g;
    P.stripe_lo = plan.stripe_lo;
    P.hull = plan.hull;
    P.halo = plan.halo;
    P.colours = colours;
    P.sweep0 = sweep0;
    P.nsweeps = nsweeps;
    P.rng = rng;
    P.xbuf = plan.xbuf;
    P.status = plan.status;
    P.ring = ring;
    P.counts = counts;
    P.burn = burn;
    P.stride = stride;
    P.epoch = epoch;
    void* args[] = {&P};
    return (int)cudaLaunchCooperativeKernel(reg_pick(plan.threads, flips != nullptr, colours != nullptr), dim3(plan.ctas), dim3(plan.threads), args,
                                            plan.smem_bytes, reinterpret_cast<cudaStream_t>(stream));
}

// This file's debug word (failures, then the id, index and bound of the
// first failed check); cudaErrorNotSupported in the normal build.
int dbg_fetch_regdom(unsigned long long* out, bool clear)
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
