// Device-side site updates shared by the kernels: Philox4x32-10, the
// heat-bath draw, and the per-lattice 128-site group update on bit-packed
// rows (global or shared memory alike).  Included by the .cu files only.
#pragma once

#include "tl_internal.h"

#include <cstdint>

namespace tl {

#define TL_DEV __device__ __forceinline__

// Bounds checks of the debug build (-DTL_DEBUG, libtiling_debug.so).  Each
// checked access asks TL_IN(i, n, id) first: an index outside [0, n) is
// counted in this translation unit's debug word (failures, then the id,
// index and bound of the first) and the access is skipped, so a wrong index
// shows up as a reported failure (tl_debug_checks) instead of a fault.  In
// the normal build the checks compile to nothing.  The ids name the check
// sites: 1xx register kernel, 2xx shared-memory resident kernel, 3xx batch
// kernel, 4xx per-pass and read-back kernels, 5xx domino shuffling.
#ifdef TL_DEBUG
static __device__ unsigned long long tl_dbg_word[4];
__device__ __noinline__ static bool tl_dbg_fail(long long i, long long n, int id)
{
    if (atomicAdd(&tl_dbg_word[0], 1ull) == 0ull) {
        tl_dbg_word[1] = (unsigned long long)id;
        tl_dbg_word[2] = (unsigned long long)i;
        tl_dbg_word[3] = (unsigned long long)n;
    }
    return false;
}
TL_DEV bool tl_in(long long i, long long n, int id) { return (i >= 0 && i < n) ? true : tl_dbg_fail(i, n, id); }
#define TL_IN(i, n, id) ::tl::tl_in((long long)(i), (long long)(n), (id))
// host side: read (and clear) this translation unit's word
static inline int tl_dbg_fetch(unsigned long long* out, bool clear)
{
    cudaError_t e = cudaMemcpyFromSymbol(out, tl_dbg_word, sizeof(unsigned long long) * 4);
    if (e == cudaSuccess && clear) {
        const unsigned long long z[4] = {0, 0, 0, 0};
        e = cudaMemcpyToSymbol(tl_dbg_word, z, sizeof(z));
    }
    return (int)e;
}
#else
#define TL_IN(i, n, id) true
#endif

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications by fixed odd constants, XOR of the high halves
// into the other two words and the round key, and a Weyl key schedule.
TL_DEV uint4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                      uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = c0 * 0xD2511F53u, hi0 = __umulhi(c0, 0xD2511F53u);
        const uint32_t lo1 = c2 * 0xCD9E8D57u, hi1 = __umulhi(c2, 0xCD9E8D57u);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

TL_DEV uint4 ld4(const uint32_t* p) { return *reinterpret_cast<const uint4*>(p); }
TL_DEV void st4(uint32_t* p, uint4 v) { *reinterpret_cast<uint4*>(p) = v; }
TL_DEV uint4 x4(uint4 a, uint4 b) { return make_uint4(a.x ^ b.x, a.y ^ b.y, a.z ^ b.z, a.w ^ b.w); }
TL_DEV bool any4(uint4 a) { return (a.x | a.y | a.z | a.w) != 0u; }
TL_DEV uint32_t popc4(uint4 a) { return __popc(a.x) + __popc(a.y) + __popc(a.z) + __popc(a.w); }

// Site j of a plane shifted by one: bit j of the result is bit j-1 (shl) or
// bit j+1 (shr) of the plane row, using the neighbouring words.
TL_DEV uint4 shl1(uint4 w, uint32_t prev)
{
    return make_uint4((w.x << 1) | (prev >> 31), (w.y << 1) | (w.x >> 31),
                      (w.z << 1) | (w.y >> 31), (w.w << 1) | (w.z >> 31));
}
TL_DEV uint4 shr1(uint4 w, uint32_t next)
{
    return make_uint4((w.x >> 1) | (w.y << 31), (w.y >> 1) | (w.z << 31),
                      (w.z >> 1) | (w.w << 31), (w.w >> 1) | (next << 31));
}

// Apply flips to a plane whose bit j-1 belongs to site j.  Words k0..k0+2
// belong to this group alone; word k0+3 shares its top bit with the next
// group and word k0-1 its top bit with this one: those two use atomicXor.
TL_DEV void store_shl(uint32_t* p, uint4 raw, uint4 fl, int k0)
{
    p[0] = raw.x ^ ((fl.x >> 1) | (fl.y << 31));
    p[1] = raw.y ^ ((fl.y >> 1) | (fl.z << 31));
    p[2] = raw.z ^ ((fl.z >> 1) | (fl.w << 31));
    if (fl.w >> 1) atomicXor(p + 3, fl.w >> 1);
    if ((fl.x & 1u) && k0 > 0) atomicXor(p - 1, 0x80000000u);
}
// Apply flips to a plane whose bit j+1 belongs to site j (mirror image).
TL_DEV void store_shr(uint32_t* p, uint4 raw, uint4 fl, int k0, int K)
{
    if (fl.x << 1) atomicXor(p, fl.x << 1);
    p[1] = raw.y ^ ((fl.y << 1) | (fl.x >> 31));
    p[2] = raw.z ^ ((fl.z << 1) | (fl.y >> 31));
    p[3] = raw.w ^ ((fl.w << 1) | (fl.z >> 31));
    if ((fl.w >> 31) && k0 + 4 < K) atomicXor(p + 4, 1u);
}

// Heat-bath draw for the flippable sites f of one group: UP iff u < t.  The
// comparison is exact and MSB first; plane k of u is one Philox output with
// counter (group, sweep, (k << 16) | pass, stream), supplied by `rnd`.  It
// stops once no flippable site is undecided, or after plane kmax, beyond
// which every remaining threshold bit is zero (so an undecided u is >= t).
TL_DEV void hb_compare(uint4& lt, uint4& und, uint4 o, uint4 t);
template <class RND, class TB>
TL_DEV uint4 heat_bath(uint4 f, int kmax, const RND& rnd, const TB& tb)
{
    uint4 und = f;
    uint4 lt = make_uint4(0u, 0u, 0u, 0u);
    // planes drawn two at a time (a plane compared after every site is
    // decided changes nothing)
    int k = 0;
    for (; k + 1 <= kmax; k += 2) {
        if (!any4(und)) return lt;
        const uint4 o0 = rnd(k), o1 = rnd(k + 1);
        const uint4 t0 = tb(k), t1 = tb(k + 1);
        hb_compare(lt, und, o0, t0);
        hb_compare(lt, und, o1, t1);
    }
    if (k <= kmax && any4(und)) hb_compare(lt, und, rnd(k), tb(k));
    return lt;
}

// Random planes computed on the spot.
struct RndPhilox {
    uint32_t grp, sweep, pass;
    DevRng rng;
    TL_DEV uint4 operator()(int k) const
    {
        return philox10(grp, sweep, ((uint32_t)k << 16) | pass, rng.stream, rng.k0, rng.k1);
    }
};
// Colour of pass slot `slot` of sweep `sweep` when the pass order is random
// (RandomWalk, Sec. 2.2, picks each step's colour at random): word 0 of the
// Philox output for counter (2^32-1, sweep, 0xFFFF0000 | slot, stream), a
// counter no site draw uses, scaled to [0, P).
TL_DEV uint32_t slot_colour(const DevRng& rng, uint32_t sweep, uint32_t slot, int P)
{
    const uint4 o = philox10(0xFFFFFFFFu, sweep, 0xFFFF0000u | slot, rng.stream, rng.k0, rng.k1);
    return (uint32_t)(((uint64_t)o.x * (uint64_t)P) >> 32);
}

// The first `npre` planes precomputed (shared memory, plane-major with
// stride `stride` uint4s), the rest computed on the spot.
struct RndPre {
    const uint4* pre;
    int npre, stride;
    RndPhilox more;
    TL_DEV uint4 operator()(int k) const { return k < npre ? pre[(size_t)k * stride] : more(k); }
};

// Same draw with the first `npre` planes read from shared memory: two loops,
// so the on-the-spot Philox of later planes is never evaluated for the
// planes that were generated ahead.
TL_DEV void hb_compare(uint4& lt, uint4& und, uint4 o, uint4 t)
{
    uint32_t d;
    d = o.x ^ t.x; lt.x |= und.x & d & t.x; und.x &= ~d;
    d = o.y ^ t.y; lt.y |= und.y & d & t.y; und.y &= ~d;
    d = o.z ^ t.z; lt.z |= und.z & d & t.z; und.z &= ~d;
    d = o.w ^ t.w; lt.w |= und.w & d & t.w; und.w &= ~d;
}
template <class TB>
TL_DEV uint4 heat_bath(uint4 f, int kmax, const RndPre& rnd, const TB& tb)
{
    uint4 und = f;
    uint4 lt = make_uint4(0u, 0u, 0u, 0u);
    const int kp = (kmax + 1) < rnd.npre ? (kmax + 1) : rnd.npre;
    int k = 0;
    // Planes are compared in small blocks whose loads and draws are issued
    // together: comparing a plane after every site is decided changes
    // nothing (the undecided mask is then zero), so only the latency of the
    // chain changes, not the result.
    for (; k + 4 <= kp; k += 4) {
        if (!any4(und)) return lt;
        const uint4 p0 = rnd.pre[(size_t)k * rnd.stride], p1 = rnd.pre[(size_t)(k + 1) * rnd.stride],
                    p2 = rnd.pre[(size_t)(k + 2) * rnd.stride], p3 = rnd.pre[(size_t)(k + 3) * rnd.stride];
        hb_compare(lt, und, p0, tb(k));
        hb_compare(lt, und, p1, tb(k + 1));
        hb_compare(lt, und, p2, tb(k + 2));
        hb_compare(lt, und, p3, tb(k + 3));
    }
    for (; k < kp; ++k) {
        if (!any4(und)) return lt;
        hb_compare(lt, und, rnd.pre[(size_t)k * rnd.stride], tb(k));
    }
    for (; k + 1 <= kmax; k += 2) {
        if (!any4(und)) return lt;
        const uint4 o0 = rnd.more(k), o1 = rnd.more(k + 1);
        hb_compare(lt, und, o0, tb(k));
        hb_compare(lt, und, o1, tb(k + 1));
    }
    if (k <= kmax && any4(und)) hb_compare(lt, und, rnd.more(k), tb(k));
    return lt;
}

struct TbScalar {
    uint32_t t;
    TL_DEV uint4 operator()(int k) const
    {
        const uint32_t b = ((t >> (31 - k)) & 1u) ? 0xFFFFFFFFu : 0u;
        return make_uint4(b, b, b, b);
    }
};
struct TbPlanes {
    const uint32_t* p;  // plane 0 of this group's four words
    int K;
    TL_DEV uint4 operator()(int k) const { return ld4(p + (size_t)k * K); }
};

// Bit-sliced 16-entry lookup: bit (31-k) of t16[idx] for each site, idx from
// its four corner bits (idx bit 0 = tl, 1 = tr, 2 = br, 3 = bl).
TL_DEV uint32_t sel_pair(uint32_t x, uint32_t tt, int q)
{
    const uint32_t a = (tt >> (2 * q)) & 1u, b = (tt >> (2 * q + 1)) & 1u;
    return ((0u - a) & ~x) | ((0u - b) & x);
}
TL_DEV uint32_t lut16(uint32_t tl, uint32_t tr, uint32_t br, uint32_t bl, uint32_t tt)
{
    if (tt == 0u) return 0u;
    if (tt == 0xFFFFu) return 0xFFFFFFFFu;
    uint32_t v[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) v[q] = sel_pair(tl, tt, q);
    uint32_t w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) w[r] = (tr & v[2 * r + 1]) | (~tr & v[2 * r]);
    const uint32_t z0 = (br & w[1]) | (~br & w[0]);
    const uint32_t z1 = (br & w[3]) | (~br & w[2]);
    return (bl & z1) | (~bl & z0);
}
// The same lookup from an expanded table: T[idx] is all ones where bit 31-k
// of t16[idx] is set, else zero (16 words per plane), so each level of the
// selection tree is one three-input bitwise select.
TL_DEV uint32_t sel(uint32_t c, uint32_t a1, uint32_t a0) { return (c & a1) | (~c & a0); }
// T must be 16-byte aligned (four vector loads).
TL_DEV uint32_t lut16_tab(uint32_t tl, uint32_t tr, uint32_t br, uint32_t bl, const uint32_t* T)
{
    const uint4* T4 = reinterpret_cast<const uint4*>(T);
    const uint4 a = T4[0], b = T4[1], c = T4[2], d = T4[3];
    const uint32_t v0 = sel(tl, a.y, a.x), v1 = sel(tl, a.w, a.z), v2 = sel(tl, b.y, b.x),
                   v3 = sel(tl, b.w, b.z), v4 = sel(tl, c.y, c.x), v5 = sel(tl, c.w, c.z),
                   v6 = sel(tl, d.y, d.x), v7 = sel(tl, d.w, d.z);
    const uint32_t w0 = sel(tr, v1, v0), w1 = sel(tr, v3, v2), w2 = sel(tr, v5, v4), w3 = sel(tr, v7, v6);
    return sel(bl, sel(br, w3, w2), sel(br, w1, w0));
}
struct TbTable {
    const uint32_t* tmask;
    const uint32_t* ttab;   // expanded table [32][16] or nullptr
    uint4 tl, tr, br, bl;
    TL_DEV uint4 operator()(int k) const
    {
        if (ttab) {
            const uint32_t* T = ttab + 16 * k;
            return make_uint4(lut16_tab(tl.x, tr.x, br.x, bl.x, T), lut16_tab(tl.y, tr.y, br.y, bl.y, T),
                              lut16_tab(tl.z, tr.z, br.z, bl.z, T), lut16_tab(tl.w, tr.w, br.w, bl.w, T));
        }
        const uint32_t tt = tmask[k];
        return make_uint4(lut16(tl.x, tr.x, br.x, bl.x, tt), lut16(tl.y, tr.y, br.y, bl.y, tt),
                          lut16(tl.z, tr.z, br.z, bl.z, tt), lut16(tl.w, tr.w, br.w, bl.w, tt));
    }
};

// Count form of the six-vertex lookup: x_i = corner bit i XOR polarity bit
// i, n = x_0 + x_1 + x_2 + x_3 in bit-sliced binary (n0, n1, n2), and the
// threshold bit of plane k is entry n of C_k = ctab + 8k (C_k[n] all ones
// where bit 31-k of t5[n] is set).  C must be 16-byte aligned.
TL_DEV void corner_count(uint32_t x0, uint32_t x1, uint32_t x2, uint32_t x3, uint32_t& n0, uint32_t& n1,
                         uint32_t& n2)
{
    const uint32_t a = x0 ^ x1, b = x0 & x1, c = x2 ^ x3, d = x2 & x3;
    const uint32_t e = a & c;        // carry of the low bits (then b = d = 0)
    n0 = a ^ c;
    n1 = b ^ d ^ e;
    n2 = b & d;                      // n = 4
}
TL_DEV uint32_t lut5(uint32_t n0, uint32_t n1, uint32_t n2, uint4 c03, uint32_t c4)
{
    return sel(n2, c4, sel(n1, sel(n0, c03.w, c03.z), sel(n0, c03.y, c03.x)));
}
struct TbCount {
    const uint32_t* ctab;   // expanded [32][8], entries 0..4 used
    uint4 n0, n1, n2;
    TL_DEV uint4 operator()(int k) const
    {
        const uint32_t* C = ctab + 8 * k;
        const uint4 c03 = *reinterpret_cast<const uint4*>(C);
        const uint32_t c4 = C[4];
        return make_uint4(lut5(n0.x, n1.x, n2.x, c03, c4), lut5(n0.y, n1.y, n2.y, c03, c4),
                          lut5(n0.z, n1.z, n2.z, c03, c4), lut5(n0.w, n1.w, n2.w, c03, c4));
    }
};
// All-ones where polarity bit i of `pol` is set.
TL_DEV uint32_t polmask(int pol, int i) { return ((pol >> i) & 1) ? 0xFFFFFFFFu : 0u; }

TL_DEV uint32_t range_mask(int k, int jlo, int jhi)
{
    int lo = jlo - 32 * k, hi = jhi - 32 * k;
    if (hi < 0 || lo > 31 || lo > hi) return 0u;
    lo = lo < 0 ? 0 : lo;
    hi = hi > 31 ? 31 : hi;
    const uint32_t mhi = (hi == 31) ? 0xFFFFFFFFu : ((1u << (hi + 1)) - 1u);
    return mhi & ~((1u << lo) - 1u);
}

// ---------------------------------------------------------------------------
// Dominoes (Sec. 1.1.3, Sec. 2.2).  Row y, class `pass`: sites x = 2j + p with
// p = (pass + y) mod 2.  Edges: E = Hz(x,y), W = Hz(x-1,y), N = Vt(x,y),
// S = Vt(x,y-1).  Planes 0 Hz_even, 1 Hz_odd, 2 Vt_even, 3 Vt_odd.
// `row` points at plane 0 of row y; RW is the row pitch in words.
// ---------------------------------------------------------------------------
template <int TK, class RND>
TL_DEV void domino_update(uint32_t* row, int64_t RW, int K, int y, int m, uint32_t pass,
                          const RND& rnd, const ThrView& th, uint32_t* nflip = nullptr)
{
    const int p = (int)((pass + (uint32_t)y) & 1u);
    const int k0 = m << 2;
    uint32_t* pE = row + (size_t)p * K + k0;
    uint32_t* pN = row + (size_t)(2 + p) * K + k0;
    uint32_t* pS = row - RW + (size_t)(2 + p) * K + k0;
    uint32_t* pHe = row + k0;
    uint32_t* pHo = row + (size_t)K + k0;
    const uint4 E = ld4(pE), N = ld4(pN), S = ld4(pS);
    uint4 Wd, Ho;
    if (p) {
        Wd = ld4(pHe);
        Ho = Wd;
    } else {
        Ho = ld4(pHo);
        Wd = shl1(Ho, k0 ? pHo[-1] : 0u);
    }
    uint4 f;
    f.x = (E.x & Wd.x & ~(N.x | S.x)) | (N.x & S.x & ~(E.x | Wd.x));
    f.y = (E.y & Wd.y & ~(N.y | S.y)) | (N.y & S.y & ~(E.y | Wd.y));
    f.z = (E.z & Wd.z & ~(N.z | S.z)) | (N.z & S.z & ~(E.z | Wd.z));
    f.w = (E.w & Wd.w & ~(N.w | S.w)) | (N.w & S.w & ~(E.w | Wd.w));
    if (!any4(f)) return;
    uint4 lt;
    if (TK == THR_SITE) {
        TbPlanes tb{th.planes + ((size_t)(y * 2 + p) * 32) * K + k0, K};
        lt = heat_bath(f, 31, rnd, tb);
    } else {
        TbScalar tb{th.scalar};
        lt = heat_bath(f, th.kmax, rnd, tb);
    }
    // a flippable site with E set is UP now; it flips iff the draw disagrees
    const uint4 fl = make_uint4(f.x & (lt.x ^ E.x), f.y & (lt.y ^ E.y), f.z & (lt.z ^ E.z),
                                f.w & (lt.w ^ E.w));
    if (!any4(fl)) return;
    if (nflip) *nflip += popc4(fl);
    st4(pE, x4(E, fl));
    st4(pN, x4(N, fl));
    st4(pS, x4(S, fl));
    if (p) st4(pHe, x4(Wd, fl));
    else store_shl(pHo, Ho, fl, k0);
}

// Single-plane fast path for dominoes with t = 2^31 (every flippable site
// goes UP iff the first random plane has a 0 there), used by the resident
// kernel.  Branch-free over the row parity p and free of atomics: the word of
// the shifted W plane that straddles two groups (bit 31 of word k0+3 when
// p = 0) is written entirely by this group, which recomputes the decision of
// the next group's first site from `onext` (bit 0 of that group's first
// random word; 0 if that group holds no domain site).  This group therefore
// never writes bit 31 of word k0-1: the group to its left does, which is why
// the planner lists one extra group left of every active range.  Because a
// group reads its neighbours' boundary words, all groups of a pass must
// finish domino_fast_compute before any of them runs domino_fast_store.
struct DominoFast {
    uint32_t* base;      // plane 0 of row y, word k0
    int64_t soff;        // offset of the S plane row relative to base
    int K, p;
    uint4 He, Ho, N, S;  // new values
    uint32_t nfl;        // sites of the group that flip
};

// `gp` points at plane 0, word k0 of the group's row.
TL_DEV DominoFast domino_fast_compute(uint32_t* gp, int64_t RW, int K, int p, int k0, uint4 o, uint32_t onext)
{
    DominoFast r;
    uint32_t* row = gp - k0;
    uint32_t* pHe = gp;
    uint32_t* pHo = gp + K;
    uint32_t* pN = gp + (size_t)(2 + p) * K;
    uint32_t* pS = gp - RW + (size_t)(2 + p) * K;
    const uint4 He = ld4(pHe), Ho = ld4(pHo), N = ld4(pN), S = ld4(pS);
    const uint32_t prev = k0 ? pHo[-1] : 0u;
    const bool more = k0 + 4 < K;
    const uint32_t eN = more ? pHe[4] : 0u;                              // Hz_e word k0+4
    const uint32_t nN = more ? row[(size_t)2 * K + k0 + 4] : 0u;         // Vt_e[y] word k0+4
    const uint32_t sN = more ? row[-RW + (int64_t)2 * K + k0 + 4] : 0u;  // Vt_e[y-1] word k0+4
    const uint4 E = p ? Ho : He;
    const uint4 Wd = p ? He : shl1(Ho, prev);
    uint4 f;
    f.x = (E.x & Wd.x & ~(N.x | S.x)) | (N.x & S.x & ~(E.x | Wd.x));
    f.y = (E.y & Wd.y & ~(N.y | S.y)) | (N.y & S.y & ~(E.y | Wd.y));
    f.z = (E.z & Wd.z & ~(N.z | S.z)) | (N.z & S.z & ~(E.z | Wd.z));
    f.w = (E.w & Wd.w & ~(N.w | S.w)) | (N.w & S.w & ~(E.w | Wd.w));
    // UP iff the plane-0 bit is 0; a flippable site flips iff that differs from E
    const uint4 fl = make_uint4(f.x & (~o.x ^ E.x), f.y & (~o.y ^ E.y), f.z & (~o.z ^ E.z), f.w & (~o.w ^ E.w));
    // the next group's first site: its W edge is bit 31 of word k0+3 (p = 0)
    const uint32_t En = eN & 1u, Wn = Ho.w >> 31, Nn = nN & 1u, Sn = sN & 1u;
    const uint32_t fn = (En & Wn & ~(Nn | Sn)) | (Nn & Sn & ~(En | Wn));
    const uint32_t fln = fn & (~onext ^ En) & 1u;
    const uint4 sh = make_uint4((fl.x >> 1) | (fl.y << 31), (fl.y >> 1) | (fl.z << 31),
                                (fl.z >> 1) | (fl.w << 31), (fl.w >> 1) | (fln << 31));
    r.nfl = popc4(fl);
    r.base = pHe;
    r.soff = -RW + (int64_t)(2 + p) * K;
    r.K = K;
    r.p = p;
    r.He = x4(He, fl);              // E when p = 0, W when p = 1
    r.Ho = x4(Ho, p ? fl : sh);     // E when p = 1, shifted W when p = 0
    r.N = x4(N, fl);
    r.S = x4(S, fl);
    return r;
}

TL_DEV void domino_fast_store(const DominoFast& r)
{
    st4(r.base, r.He);
    st4(r.base + r.K, r.Ho);
    st4(r.base + (size_t)(2 + r.p) * r.K, r.N);
    st4(r.base + r.soff, r.S);
}

// ---------------------------------------------------------------------------
// Lozenges (Sec. 1.2.1).  Row y, class `pass`: sites x = 3j + r with
// r = (pass - y) mod 3.  Six edges in angular order e0 = E1(x,y),
// e1 = E3(x,y), e2 = E2(x,y), e3 = E1(x-1,y), e4 = E3(x-1,y-1),
// e5 = E2(x,y-1); UP (cube present) = {e0,e2,e4}, DOWN = {e1,e3,e5}.
// Planes: E1_r = r, E2_r = 3 + r, E3_r = 6 + r.
// ---------------------------------------------------------------------------
template <int TK, class RND>
TL_DEV void lozenge_update(uint32_t* row, int64_t RW, int K, int y, int m, uint32_t pass,
                           const RND& rnd, const ThrView& th, uint32_t* nflip = nullptr)
{
    const int r = (int)((pass + 3u - (uint32_t)(y % 3)) % 3u);
    const int k0 = m << 2;
    uint32_t* dn = row - RW;
    uint32_t* p0 = row + (size_t)r * K + k0;
    uint32_t* p1 = row + (size_t)(6 + r) * K + k0;
    uint32_t* p2 = row + (size_t)(3 + r) * K + k0;
    uint32_t* p5 = dn + (size_t)(3 + r) * K + k0;
    uint32_t *p3, *p4;
    const uint4 e0 = ld4(p0), e1 = ld4(p1), e2 = ld4(p2), e5 = ld4(p5);
    uint4 e3, e4, raw3, raw4;
    if (r) {
        p3 = row + (size_t)(r - 1) * K + k0;
        p4 = dn + (size_t)(6 + r - 1) * K + k0;
        e3 = raw3 = ld4(p3);
        e4 = raw4 = ld4(p4);
    } else {
        p3 = row + (size_t)2 * K + k0;
        p4 = dn + (size_t)8 * K + k0;
        raw3 = ld4(p3);
        raw4 = ld4(p4);
        e3 = shl1(raw3, k0 ? p3[-1] : 0u);
        e4 = shl1(raw4, k0 ? p4[-1] : 0u);
    }
    uint4 f;
#define TL_LOZ_F(c) ((e0.c & e2.c & e4.c & ~(e1.c | e3.c | e5.c)) | (e1.c & e3.c & e5.c & ~(e0.c | e2.c | e4.c)))
    f.x = TL_LOZ_F(x); f.y = TL_LOZ_F(y); f.z = TL_LOZ_F(z); f.w = TL_LOZ_F(w);
#undef TL_LOZ_F
    if (!any4(f)) return;
    uint4 lt;
    if (TK == THR_SITE) {
        TbPlanes tb{th.planes + ((size_t)(y * 3 + r) * 32) * K + k0, K};
        lt = heat_bath(f, 31, rnd, tb);
    } else {
        TbScalar tb{th.scalar};
        lt = heat_bath(f, th.kmax, rnd, tb);
    }
    const uint4 fl = make_uint4(f.x & (lt.x ^ e0.x), f.y & (lt.y ^ e0.y), f.z & (lt.z ^ e0.z),
                                f.w & (lt.w ^ e0.w));
    if (!any4(fl)) return;
    if (nflip) *nflip += popc4(fl);
    st4(p0, x4(e0, fl));
    st4(p1, x4(e1, fl));
    st4(p2, x4(e2, fl));
    st4(p5, x4(e5, fl));
    if (r) {
        st4(p3, x4(raw3, fl));
        st4(p4, x4(raw4, fl));
    } else {
        store_shl(p3, raw3, fl, k0);
        store_shl(p4, raw4, fl, k0);
    }
}

// ---------------------------------------------------------------------------
// Six-vertex faces (Sec. 1.2.4, Fig. 5C).  Face row Y (vertex rows Y, Y+1),
// class (px, py) from the pass order (0,0),(1,1),(1,0),(0,1): faces
// X = 2j + px.  B = Hz(X,Y), T = Hz(X,Y+1), L = Vt(X,Y), R = Vt(X+1,Y);
// corner bits TL = Vt(X,Y+1), TR = Hz(X+1,Y+1), BR = Hz(X+1,Y),
// BL = Hz(X-1,Y).  UP = path through B and L.  Interior faces only.
// ---------------------------------------------------------------------------
TL_DEV int sixv_px(uint32_t pass) { return (pass == 1u || pass == 2u) ? 1 : 0; }
TL_DEV int sixv_py(uint32_t pass) { return (pass == 1u || pass == 3u) ? 1 : 0; }

template <class RND>
TL_DEV void sixv_update(uint32_t* row, int64_t RW, int K, int N, int Y, int m, uint32_t pass,
                        const RND& rnd, const ThrView& th, const uint32_t* ttab, const uint32_t* ctab,
                        uint32_t* nflip = nullptr)
{
    const int px = sixv_px(pass);
    const int k0 = m << 2;
    uint32_t* up = row + RW;
    uint32_t *pB, *pT, *pL, *pR;
    uint4 B, T, L, R, TL, TR, BR, BL, rawR;
    if (px == 0) {
        pB = row + k0;
        pT = up + k0;
        pL = row + (size_t)2 * K + k0;
        pR = row + (size_t)3 * K + k0;
        B = ld4(pB); T = ld4(pT); L = ld4(pL); R = rawR = ld4(pR);
        BR = ld4(row + (size_t)K + k0);
        TR = ld4(up + (size_t)K + k0);
        TL = ld4(up + (size_t)2 * K + k0);
        BL = shl1(BR, k0 ? row[(size_t)K + k0 - 1] : 0u);
    } else {
        pB = row + (size_t)K + k0;
        pT = up + (size_t)K + k0;
        pL = row + (size_t)3 * K + k0;
        pR = row + (size_t)2 * K + k0;
        B = ld4(pB); T = ld4(pT); L = ld4(pL);
        TL = ld4(up + (size_t)3 * K + k0);
        BL = ld4(row + k0);
        const bool more = k0 + 4 < K;
        BR = shr1(BL, more ? row[k0 + 4] : 0u);
        TR = shr1(ld4(up + k0), more ? up[k0 + 4] : 0u);
        rawR = ld4(pR);
        R = shr1(rawR, more ? pR[4] : 0u);
    }
    const int jlo = px ? 0 : 1;
    const int jhi = (N - 1 - px) >> 1;
    uint4 f;
#define TL_6V_F(c, i) (((B.c & L.c & ~(R.c | T.c)) | (R.c & T.c & ~(B.c | L.c))) & range_mask(k0 + i, jlo, jhi))
    f.x = TL_6V_F(x, 0); f.y = TL_6V_F(y, 1); f.z = TL_6V_F(z, 2); f.w = TL_6V_F(w, 3);
#undef TL_6V_F
    if (!any4(f)) return;
    uint4 lt;
    if (ctab) {
        const uint32_t p0 = polmask(th.cpol, 0), p1 = polmask(th.cpol, 1), p2 = polmask(th.cpol, 2),
                       p3 = polmask(th.cpol, 3);
        TbCount tb;
        tb.ctab = ctab;
        corner_count(TL.x ^ p0, TR.x ^ p1, BR.x ^ p2, BL.x ^ p3, tb.n0.x, tb.n1.x, tb.n2.x);
        corner_count(TL.y ^ p0, TR.y ^ p1, BR.y ^ p2, BL.y ^ p3, tb.n0.y, tb.n1.y, tb.n2.y);
        corner_count(TL.z ^ p0, TR.z ^ p1, BR.z ^ p2, BL.z ^ p3, tb.n0.z, tb.n1.z, tb.n2.z);
        corner_count(TL.w ^ p0, TR.w ^ p1, BR.w ^ p2, BL.w ^ p3, tb.n0.w, tb.n1.w, tb.n2.w);
        lt = heat_bath(f, 31, rnd, tb);
    } else {
        TbTable tb{th.tmask, ttab, TL, TR, BR, BL};
        lt = heat_bath(f, 31, rnd, tb);
    }
    const uint4 fl = make_uint4(f.x & (lt.x ^ B.x), f.y & (lt.y ^ B.y), f.z & (lt.z ^ B.z),
                                f.w & (lt.w ^ B.w));
    if (!any4(fl)) return;
    if (nflip) *nflip += popc4(fl);
    st4(pB, x4(B, fl));
    st4(pT, x4(T, fl));
    st4(pL, x4(L, fl));
    if (px == 0) st4(pR, x4(rawR, fl));
    else store_shr(pR, rawR, fl, k0, K);
}


// Dispatch one group update for lattice LAT.
// `ttab`: expanded six-vertex table in shared memory, or nullptr; `ctab`:
// expanded count table (used instead when not nullptr).  `nflip`, if not
// nullptr, is increased by the number of sites that flipped.
template <int LAT, int TK, class RND>
TL_DEV void group_update(uint32_t* row, int64_t RW, const Geom& g, int y, int m, uint32_t pass,
                         const RND& rnd, const ThrView& th, const uint32_t* ttab = nullptr,
                         const uint32_t* ctab = nullptr, uint32_t* nflip = nullptr)
{
    if (LAT == LAT_DOMINO) domino_update<TK>(row, RW, g.K, y, m, pass, rnd, th, nflip);
    else if (LAT == LAT_LOZENGE) lozenge_update<TK>(row, RW, g.K, y, m, pass, rnd, th, nflip);
    else sixv_update(row, RW, g.K, g.N, y, m, pass, rnd, th, ttab, ctab, nflip);
}

// splitmix64 output for state x (Steele, Lea & Flood 2014).
TL_DEV uint64_t mix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Hash contribution of the set bits of one packed word (row y, plane pl,
// word k) to the order-independent state hash.
TL_DEV uint64_t word_hash(uint32_t w, const Geom& g, int y, int pl, int k)
{
    const int type = pl / g.npar, res = pl - type * g.npar;
    const uint64_t base = ((uint64_t)type * g.H + y) * (uint64_t)g.W;
    uint64_t acc = 0;
    while (w) {
        const int b = __ffs(w) - 1;
        w &= w - 1;
        const int x = g.npar * (32 * k + b) + res;
        if (x < g.W) acc += mix64(base + (uint64_t)x);
    }
    return acc;
}

// Edge-occupancy counters, bit-sliced in the packed layout: counter bit b
// of the 32 edges of packed word i (row-major over the H real rows) is bit
// of word cplanes[b * H * row_words + i].  Adding a word of the state is a
// ripple-carry add over the planes that stops when no carry is left.
TL_DEV void word_count_sliced(uint32_t w, int64_t i, int64_t plane_words, uint32_t* cplanes)
{
    uint32_t carry = w;
    for (int b = 0; b < 32 && carry; ++b) {
        uint32_t* p = cplanes + (int64_t)b * plane_words + i;
        const uint32_t c = *p;
        *p = c ^ carry;
        carry &= c;
    }
}

// The same add for four consecutive words (index i a multiple of 4): one
// 16-byte read and write per counter plane, the four carries rippling
// together, so a thread's counter update is one chain of dependent accesses
// per four words instead of per word.
TL_DEV void word_count_sliced4(uint4 w, int64_t i, int64_t plane_words, uint32_t* cplanes)
{
#ifdef TL_DEBUG
    if (!TL_IN(i + 3, plane_words, 107)) return;
#endif
    uint4 carry = w;
    for (int b = 0; b < 32 && any4(carry); ++b) {
        uint4* p = reinterpret_cast<uint4*>(cplanes + (int64_t)b * plane_words + i);
        const uint4 c = *p;
        *p = x4(c, carry);
        carry = make_uint4(carry.x & c.x, carry.y & c.y, carry.z & c.z, carry.w & c.w);
    }
}

}  // namespace tl
