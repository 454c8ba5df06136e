/*
 * oracle.c -- plain, slow, single-threaded CPU oracle for colour-class
 * parallel heat-bath Glauber dynamics on domino tilings, lozenge tilings and
 * the six-vertex model (Keating & Sridhar, "Random Tilings with the GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this code.  It shares nothing
 * with the CUDA path: its own Philox, its own lattice geometry, its own
 * threshold arithmetic, its own hash.
 *
 * Canonical state (the interchange format both sides agree on):
 *   one uint8 per lattice edge, 0 or 1, laid out [plane][y][x] over a vertex
 *   box of W x H.
 *   - Domino (Sec. 1.1): plane 0 = Hz(x,y), the primal edge (x,y)-(x+1,y);
 *     plane 1 = Vt(x,y), the primal edge (x,y)-(x,y+1).  1 means a domino
 *     crosses the edge (Sec. 2.2 "tilestate" bits, stored once per edge).
 *   - Lozenge (Sec. 1.2.1): triangular lattice in axial coordinates with
 *     neighbours +-(1,0), +-(0,1), +-(1,1); plane 0 = E1(x,y) to (x+1,y),
 *     plane 1 = E2(x,y) to (x,y+1), plane 2 = E3(x,y) to (x+1,y+1).
 *     1 means the edge is the short diagonal of a lozenge.
 *   - Six-vertex (Sec. 1.2.4): box (N+2)^2 with the model's vertices at
 *     1..N; plane 0 = Hz(X,Y) east of (X,Y), plane 1 = Vt(X,Y) north of
 *     (X,Y); 1 means occupied.  External half-edges are Hz(0,Y), Hz(N,Y),
 *     Vt(X,0), Vt(X,N).
 *
 * Randomness (counter-based; the paper used TinyMT per vertex, Sec. 2.2.1):
 *   u_v is a 32-bit number whose bit (31-k) is bit (rank&31) of output word
 *   ((rank>>5)&3) of Philox4x32-10 with key (seed_lo, seed_hi) and counter
 *   (rank>>7, sweep, (k<<16)|pass, stream).  rank = r*Rp + j with the
 *   per-lattice (r, j) of the site and Rp = j-range rounded up to 128.
 *   Heat-bath: a flippable site goes UP iff u_v < t_v, else DOWN.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define OR_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as  */
/* easy as 1, 2, 3" (SC'11).  Ten rounds; each round multiplies counter     */
/* words 0 and 2 by fixed odd constants (64-bit product split hi/lo), XORs  */
/* the high halves with the other counter words and the round key, and     */
/* bumps the key by the Weyl constants between rounds.                      */
/* ------------------------------------------------------------------------ */
OR_EXPORT void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                                uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* u_v for one site, built from all 32 planes (MSB first).  A one-entry     */
/* cache keeps the 32 Philox outputs of the last 128-site group, so that a  */
/* raster walk over a row does not recompute them 128 times.                */
typedef struct {
    int valid;
    uint64_t seed;
    uint32_t stream, sweep, pass, group;
    uint32_t words[32][4];
} u_cache;

static uint32_t site_u(u_cache* cache, uint64_t seed, uint32_t stream,
                       uint32_t sweep, uint32_t pass, uint64_t rank)
{
    uint32_t group = (uint32_t)(rank >> 7);
    uint32_t word = (uint32_t)((rank >> 5) & 3u);
    uint32_t bit = (uint32_t)(rank & 31u);
    if (!cache->valid || cache->seed != seed || cache->stream != stream ||
        cache->sweep != sweep || cache->pass != pass || cache->group != group) {
        uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
        for (uint32_t k = 0; k < 32; ++k) {
            uint32_t ctr[4] = {group, sweep, (k << 16) | pass, stream};
            or_philox4x32_10(ctr, key, cache->words[k]);
        }
        cache->valid = 1; cache->seed = seed; cache->stream = stream;
        cache->sweep = sweep; cache->pass = pass; cache->group = group;
    }
    uint32_t u = 0;
    for (uint32_t k = 0; k < 32; ++k)
        u |= ((cache->words[k][word] >> bit) & 1u) << (31u - k);
    return u;
}

OR_EXPORT uint32_t or_site_u(uint64_t seed, uint32_t stream, uint32_t sweep,
                             uint32_t pass, uint64_t rank)
{
    u_cache c; c.valid = 0;
    return site_u(&c, seed, stream, sweep, pass, rank);
}

static uint64_t round_up_128(uint64_t v) { return (v + 127u) & ~(uint64_t)127u; }

/* ------------------------------------------------------------------------ */
/* State hash: order-independent sum over set edge bits of splitmix64 of    */
/* the bit's canonical linear index (Steele, Lea & Flood 2014 mixer).       */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

OR_EXPORT uint64_t or_splitmix64(uint64_t x) { return splitmix64(x); }

/* Random pass order (the RandomWalk of Sec. 2.2 picks the colour of every  */
/* step at random): slot i of sweep s visits colour floor(P w / 2^32), w =  */
/* word 0 of Philox4x32-10 with counter (2^32-1, s, 0xFFFF0000 | i, stream) */
/* (a counter no site draw uses).  The site draws of that slot are keyed    */
/* by the slot i, so two slots of one sweep on the same colour use fresh    */
/* numbers.                                                                 */
OR_EXPORT int or_slot_colour(uint64_t seed, uint32_t stream, uint32_t sweep, int slot, int P)
{
    uint32_t ctr[4] = {0xFFFFFFFFu, sweep, 0xFFFF0000u | (uint32_t)slot, stream};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    or_philox4x32_10(ctr, key, out);
    return (int)(((uint64_t)out[0] * (uint64_t)P) >> 32);
}



OR_EXPORT uint64_t or_state_hash(const uint8_t* st, uint64_t nbits)
{
    uint64_t h = 0;
    for (uint64_t i = 0; i < nbits; ++i)
        if (st[i]) h += splitmix64(i);
    return h;
}

/* ======================================================================== */
/* Domino tilings (Sec. 1.1, Sec. 2.2)                                      */
/* ======================================================================== */
#define DHZ(st, W, H, x, y) (st)[(size_t)(y) * (W) + (x)]
#define DVT(st, W, H, x, y) (st)[(size_t)(H) * (W) + (size_t)(y) * (W) + (x)]

static int dget_h(const uint8_t* st, int W, int H, int x, int y)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 0;
    return DHZ(st, W, H, x, y);
}
static int dget_v(const uint8_t* st, int W, int H, int x, int y)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 0;
    return DVT(st, W, H, x, y);
}

/* Aztec diamond of order n: faces whose centres satisfy                    */
/* |cx - n| + |cy - n| <= n; vertex box (2n+1)^2.  Initial tiling: every   */
/* row of faces covered by horizontal dominoes from its left end.           */
OR_EXPORT int or_domino_aztec_init(int n, uint8_t* st)
{
    int W = 2 * n + 1, H = 2 * n + 1;
    memset(st, 0, (size_t)2 * W * H);
    for (int y = 0; y < 2 * n; ++y) {
        int m = (y + 1 < 2 * n - y) ? (y + 1) : (2 * n - y);
        int x0 = n - m;
        for (int i = 0; i < m; ++i) {
            int left = x0 + 2 * i;
            /* the domino covers faces (left,y),(left+1,y): it crosses the  */
            /* vertical primal edge (left+1,y)-(left+1,y+1).                */
            DVT(st, W, H, left + 1, y) = 1;
        }
    }
    return 0;
}

/* Rectangle of w x h faces; vertex box (w+1) x (h+1).  All-horizontal if  */
/* w is even, else all-vertical if h is even, else not tileable (-1).      */
OR_EXPORT int or_domino_rect_init(int w, int h, uint8_t* st)
{
    int W = w + 1, H = h + 1;
    memset(st, 0, (size_t)2 * W * H);
    if (w % 2 == 0) {
        for (int y = 0; y < h; ++y)
            for (int x = 0; x < w; x += 2) DVT(st, W, H, x + 1, y) = 1;
        return 0;
    }
    if (h % 2 == 0) {
        for (int y = 0; y < h; y += 2)
            for (int x = 0; x < w; ++x) DHZ(st, W, H, x, y + 1) = 1;
        return 0;
    }
    return -1;
}

/* Site state at vertex (x,y): 2 = UP (two vertical dominoes: E and W      */
/* edges crossed, tilestate 12), 1 = DOWN (two horizontal dominoes: N and  */
/* S crossed, tilestate 3), 0 = not rotatable (Sec. 2.2).                   */
static int domino_site_state(const uint8_t* st, int W, int H, int x, int y)
{
    int e = dget_h(st, W, H, x, y), w = dget_h(st, W, H, x - 1, y);
    int n = dget_v(st, W, H, x, y), s = dget_v(st, W, H, x, y - 1);
    if (e && w && !n && !s) return 2;
    if (n && s && !e && !w) return 1;
    return 0;
}

static void domino_site_set(uint8_t* st, int W, int H, int x, int y, int up)
{
    DHZ(st, W, H, x, y) = (uint8_t)up;
    DHZ(st, W, H, x - 1, y) = (uint8_t)up;
    DVT(st, W, H, x, y) = (uint8_t)!up;
    DVT(st, W, H, x, y - 1) = (uint8_t)!up;
}

/* Colour class of a domino site: (x + y) mod 2 (Sec. 1.1.3). */
OR_EXPORT void or_domino_site_states(const uint8_t* st, int W, int H, int pass,
                                     uint8_t* out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            out[(size_t)y * W + x] = (((x + y) & 1) == pass)
                                         ? (uint8_t)domino_site_state(st, W, H, x, y)
                                         : 0;
}

/* Cluster rotation over one colour class with given decisions: every      */
/* rotatable class site goes UP where dec=1, DOWN where dec=0.             */
OR_EXPORT void or_domino_apply_pass(uint8_t* st, int W, int H, int pass,
                                    const uint8_t* dec)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            if (((x + y) & 1) != pass) continue;
            if (domino_site_state(st, W, H, x, y) == 0) continue;
            domino_site_set(st, W, H, x, y, dec[(size_t)y * W + x] ? 1 : 0);
        }
}

OR_EXPORT int or_domino_sweeps(uint8_t* st, int W, int H,
                               const uint32_t* t_site, uint32_t t_scalar,
                               uint64_t seed, uint32_t stream, uint64_t sweep0,
                               uint64_t nsweeps, uint64_t* hashes, int random_order)
{
    uint64_t Rp = round_up_128((uint64_t)(W + 1) / 2);
    uint8_t* dec = (uint8_t*)calloc((size_t)W * H, 1);
    if (!dec) return -1;
    u_cache cache; cache.valid = 0;
    for (uint64_t s = sweep0; s < sweep0 + nsweeps; ++s) {
        for (int slot = 0; slot < 2; ++slot) {
            const int pass = random_order ? or_slot_colour(seed, stream, (uint32_t)s, slot, 2) : slot;
            /* draw the decisions for every rotatable site of the class ... */
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    size_t i = (size_t)y * W + x;
                    dec[i] = 0;
                    if (((x + y) & 1) != pass) continue;
                    if (domino_site_state(st, W, H, x, y) == 0) continue;
                    uint64_t rank = (uint64_t)y * Rp + (uint64_t)(x >> 1);
                    uint32_t u = site_u(&cache, seed, stream, (uint32_t)s,
                                        (uint32_t)slot, rank);
                    uint32_t t = t_site ? t_site[i] : t_scalar;
                    dec[i] = (u < t) ? 1 : 0;
                }
            /* ... then rotate the whole cluster at once (Eq. 1.1). */
            or_domino_apply_pass(st, W, H, pass, dec);
        }
        if (hashes) hashes[s - sweep0] = or_state_hash(st, (uint64_t)2 * W * H);
    }
    free(dec);
    return 0;
}

/* Heat-bath thresholds from dual-edge weights (Sec. 1.1.1): at a site,    */
/* P(UP) = wE*wW / (wE*wW + wN*wS) with the weights of the four primal     */
/* edges around it (edges outside the box weigh 1).  t = floor(P * 2^32), */
/* clamped to 2^32-1.  w is laid out like the canonical state.              */
static double dw_h(const double* w, int W, int H, int x, int y)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 1.0;
    return w[(size_t)y * W + x];
}
static double dw_v(const double* w, int W, int H, int x, int y)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 1.0;
    return w[(size_t)H * W + (size_t)y * W + x];
}

static uint32_t prob_to_threshold(double p)
{
    double t = floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 0xFFFFFFFFu;
    if (t <= 0.0) return 0u;
    return (uint32_t)t;
}

OR_EXPORT void or_domino_thresholds(const double* w, int W, int H, uint32_t* t)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            double we = dw_h(w, W, H, x, y), ww = dw_h(w, W, H, x - 1, y);
            double wn = dw_v(w, W, H, x, y), ws = dw_v(w, W, H, x, y - 1);
            double up = we * ww;
            double down = wn * ws;
            t[(size_t)y * W + x] = prob_to_threshold(up / (up + down));
        }
}

/* W(T) = product over dominoes of their dual-edge weight (Sec. 1.1.1).    */
OR_EXPORT double or_domino_weight(const uint8_t* st, int W, int H, const double* w)
{
    double prod = 1.0;
    for (size_t i = 0; i < (size_t)2 * W * H; ++i)
        if (st[i]) prod *= w[i];
    return prod;
}

/* Faces of the domain are recovered from a tiling: face (x,y) (lower-left */
/* corner (x,y)) is covered iff exactly one of its four edges is crossed.  */
static int domino_face_cover(const uint8_t* st, int W, int H, int x, int y)
{
    return dget_h(st, W, H, x, y) + dget_h(st, W, H, x, y + 1) +
           dget_v(st, W, H, x, y) + dget_v(st, W, H, x + 1, y);
}

/* Validity: every face is covered at most once, and the covered faces are */
/* exactly the given face mask ([H-1][W-1], 1 = face in the domain).       */
/* Returns the number of violations.                                        */
OR_EXPORT int64_t or_domino_check(const uint8_t* st, int W, int H,
                                  const uint8_t* face_mask)
{
    int64_t bad = 0;
    for (int y = 0; y < H - 1; ++y)
        for (int x = 0; x < W - 1; ++x) {
            int c = domino_face_cover(st, W, H, x, y);
            int want = face_mask ? face_mask[(size_t)y * (W - 1) + x] : (c > 0);
            if (c > 1 || c != want) ++bad;
        }
    /* no crossed edge may lie on the box border */
    for (int y = 0; y < H; ++y) if (DHZ(st, W, H, W - 1, y)) ++bad;
    for (int x = 0; x < W; ++x) if (DVT(st, W, H, x, H - 1)) ++bad;
    return bad;
}

/* Height function (Sec. 1.1, Fig. 2): h = 0 at the first domain vertex in */
/* (y, x) order; along an edge not crossed by a domino the height changes  */
/* by +1 if the face on the left of the step is black (x+y even for the    */
/* face with lower-left corner (x,y)) and -1 if white; across a crossed    */
/* edge by -3 times that.  Propagated by breadth-first search over the     */
/* edges of domain faces; returns the number of inconsistencies found.     */
/* Vertices off the domain get INT32_MIN.                                   */
#define HNONE INT32_MIN
OR_EXPORT int64_t or_domino_height(const uint8_t* st, int W, int H, int32_t* h)
{
    size_t nv = (size_t)W * H;
    uint8_t* face = (uint8_t*)calloc((size_t)W * H, 1);
    int* queue = (int*)malloc(sizeof(int) * nv);
    if (!face || !queue) { free(face); free(queue); return -1; }
    for (size_t i = 0; i < nv; ++i) h[i] = HNONE;
    for (int y = 0; y < H - 1; ++y)
        for (int x = 0; x < W - 1; ++x)
            face[(size_t)y * W + x] = domino_face_cover(st, W, H, x, y) == 1;
#define FACE(x, y) (((x) >= 0 && (y) >= 0 && (x) < W - 1 && (y) < H - 1) ? face[(size_t)(y) * W + (x)] : 0)
    int start = -1;
    for (int y = 0; y < H && start < 0; ++y)
        for (int x = 0; x < W && start < 0; ++x)
            if (FACE(x, y) || FACE(x - 1, y) || FACE(x, y - 1) || FACE(x - 1, y - 1))
                start = y * W + x;
    int64_t bad = 0;
    if (start < 0) { free(face); free(queue); return 0; }
    size_t qh = 0, qt = 0;
    h[start] = 0; queue[qt++] = start;
    while (qh < qt) {
        int v = queue[qh++];
        int x = v % W, y = v / W;
        /* four steps: +x, -x, +y, -y */
        for (int d = 0; d < 4; ++d) {
            int nx = x, ny = y, dom, crossed, black_left;
            if (d == 0) {          /* (x,y) -> (x+1,y); left face (x,y) */
                nx = x + 1; dom = FACE(x, y) || FACE(x, y - 1);
                crossed = dget_h(st, W, H, x, y); black_left = ((x + y) & 1) == 0;
            } else if (d == 1) {   /* (x,y) -> (x-1,y); left face (x-1,y-1) */
                nx = x - 1; dom = FACE(x - 1, y) || FACE(x - 1, y - 1);
                crossed = dget_h(st, W, H, x - 1, y); black_left = ((x - 1 + y - 1) & 1) == 0;
            } else if (d == 2) {   /* (x,y) -> (x,y+1); left face (x-1,y) */
                ny = y + 1; dom = FACE(x - 1, y) || FACE(x, y);
                crossed = dget_v(st, W, H, x, y); black_left = ((x - 1 + y) & 1) == 0;
            } else {               /* (x,y) -> (x,y-1); left face (x,y-1) */
                ny = y - 1; dom = FACE(x - 1, y - 1) || FACE(x, y - 1);
                crossed = dget_v(st, W, H, x, y - 1); black_left = ((x + y - 1) & 1) == 0;
            }
            if (!dom) continue;
            int sgn = black_left ? 1 : -1;
            int32_t nh = h[v] + (crossed ? -3 * sgn : sgn);
            int nv_ = ny * W + nx;
            if (h[nv_] == HNONE) { h[nv_] = nh; queue[qt++] = nv_; }
            else if (h[nv_] != nh) ++bad;
        }
    }
#undef FACE
    free(face); free(queue);
    return bad;
}

/* Domino types for the arctic-circle pictures (Sec. 4).  The paper does   */
/* not fix the labels; the reading used here: a horizontal domino is north */
/* iff its left square has colour (x+y) mod 2 == kappa, a vertical domino  */
/* is west iff its bottom square has colour (x+y) mod 2 != kappa, with     */
/* kappa = n mod 2 for the Aztec diamond of order n (so the all-horizontal */
/* start is north in the upper half of the diamond).  Walks the dominoes   */
/* (crossed edges) and adds one to the type counter of both squares each   */
/* covers: counts[t][y][x] for faces (x,y), t = 0 N, 1 S, 2 E, 3 W, shape  */
/* [4][H-1][W-1].                                                           */
OR_EXPORT void or_domino_nsew(const uint8_t* st, int W, int H, int kappa, uint32_t* counts)
{
    size_t nf = (size_t)(W - 1) * (H - 1);
#define NSEW_ADD(t, fx, fy) counts[(size_t)(t) * nf + (size_t)(fy) * (W - 1) + (fx)] += 1
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            /* Vt(x,y) crossed: horizontal domino on faces (x-1,y), (x,y) */
            if (DVT(st, W, H, x, y) && x >= 1 && x < W - 1 && y < H - 1) {
                int left_colour = ((x - 1) + y) & 1;
                int t = (left_colour == kappa) ? 0 : 1;
                NSEW_ADD(t, x - 1, y);
                NSEW_ADD(t, x, y);
            }
            /* Hz(x,y) crossed: vertical domino on faces (x,y-1), (x,y) */
            if (DHZ(st, W, H, x, y) && y >= 1 && y < H - 1 && x < W - 1) {
                int bottom_colour = (x + (y - 1)) & 1;
                int t = (bottom_colour != kappa) ? 3 : 2;
                NSEW_ADD(t, x, y - 1);
                NSEW_ADD(t, x, y);
            }
        }
#undef NSEW_ADD
}

/* ======================================================================== */
/* Lozenge tilings (Sec. 1.2.1)                                             */
/* ======================================================================== */
#define LE(st, W, H, k, x, y) (st)[(size_t)(k) * (H) * (W) + (size_t)(y) * (W) + (x)]
static int lget(const uint8_t* st, int W, int H, int k, int x, int y)
{
    if (x < 0 || y < 0 || x >= W || y >= H) return 0;
    return LE(st, W, H, k, x, y);
}

/* Hexagon with sides a, b, c as the boundary of an a x b x c box of cubes  */
/* seen along (1,1,1).  A lattice point (i,j,k) projects to the axial      */
/* vertex (i-k+c, j-k+c); the box is (a+c+1) x (b+c+1).  Start: the empty  */
/* box -- floor faces (normal e3) cross E3, wall faces x=0 (normal e1)      */
/* cross E1 and wall faces y=0 (normal e2) cross E2 at their short          */
/* diagonals.                                                               */
OR_EXPORT int or_lozenge_hexagon_init(int a, int b, int c, uint8_t* st)
{
    int W = a + c + 1, H = b + c + 1;
    memset(st, 0, (size_t)3 * W * H);
    for (int i = 0; i < a; ++i)
        for (int j = 0; j < b; ++j) LE(st, W, H, 2, i + c, j + c) = 1;
    for (int j = 0; j < b; ++j)
        for (int k = 0; k < c; ++k) LE(st, W, H, 0, c - k - 1, j - k + c) = 1;
    for (int i = 0; i < a; ++i)
        for (int k = 0; k < c; ++k) LE(st, W, H, 1, i - k + c, c - k - 1) = 1;
    return 0;
}

/* The six edges around a triangular-lattice vertex v = (x,y), in angular  */
/* order: e0 = E1(x,y), e1 = E3(x,y), e2 = E2(x,y), e3 = E1(x-1,y),        */
/* e4 = E3(x-1,y-1), e5 = E2(x,y-1).  The three lozenges around v form a   */
/* hexagon (v rotatable) iff e0,e2,e4 are crossed and e1,e3,e5 are not     */
/* (a cube with corner at v can be removed: UP) or the reverse (a cube can */
/* be added: DOWN).                                                          */
static int lozenge_site_state(const uint8_t* st, int W, int H, int x, int y)
{
    int e0 = lget(st, W, H, 0, x, y), e1 = lget(st, W, H, 2, x, y);
    int e2 = lget(st, W, H, 1, x, y), e3 = lget(st, W, H, 0, x - 1, y);
    int e4 = lget(st, W, H, 2, x - 1, y - 1), e5 = lget(st, W, H, 1, x, y - 1);
    if (e0 && e2 && e4 && !e1 && !e3 && !e5) return 2;
    if (e1 && e3 && e5 && !e0 && !e2 && !e4) return 1;
    return 0;
}

static void lozenge_site_set(uint8_t* st, int W, int H, int x, int y, int up)
{
    LE(st, W, H, 0, x, y) = (uint8_t)up;
    LE(st, W, H, 1, x, y) = (uint8_t)up;
    LE(st, W, H, 2, x - 1, y - 1) = (uint8_t)up;
    LE(st, W, H, 2, x, y) = (uint8_t)!up;
    LE(st, W, H, 0, x - 1, y) = (uint8_t)!up;
    LE(st, W, H, 1, x, y - 1) = (uint8_t)!up;
}

/* Three-colouring of the triangular lattice: class (x + y) mod 3. */
OR_EXPORT void or_lozenge_site_states(const uint8_t* st, int W, int H, int pass,
                                      uint8_t* out)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            out[(size_t)y * W + x] = ((x + y) % 3 == pass)
                                         ? (uint8_t)lozenge_site_state(st, W, H, x, y)
                                         : 0;
}

OR_EXPORT void or_lozenge_apply_pass(uint8_t* st, int W, int H, int pass,
                                     const uint8_t* dec)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            if ((x + y) % 3 != pass) continue;
            if (lozenge_site_state(st, W, H, x, y) == 0) continue;
            lozenge_site_set(st, W, H, x, y, dec[(size_t)y * W + x] ? 1 : 0);
        }
}

/* t_site may be NULL (then t_scalar, the add-a-cube threshold, is used). */
OR_EXPORT int or_lozenge_sweeps(uint8_t* st, int W, int H,
                                const uint32_t* t_site, uint32_t t_scalar,
                                uint64_t seed, uint32_t stream, uint64_t sweep0,
                                uint64_t nsweeps, uint64_t* hashes, int random_order)
{
    uint64_t Rp = round_up_128((uint64_t)(W + 2) / 3);
    uint8_t* dec = (uint8_t*)calloc((size_t)W * H, 1);
    if (!dec) return -1;
    u_cache cache; cache.valid = 0;
    for (uint64_t s = sweep0; s < sweep0 + nsweeps; ++s) {
        for (int slot = 0; slot < 3; ++slot) {
            const int pass = random_order ? or_slot_colour(seed, stream, (uint32_t)s, slot, 3) : slot;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    size_t i = (size_t)y * W + x;
                    dec[i] = 0;
                    if ((x + y) % 3 != pass) continue;
                    if (lozenge_site_state(st, W, H, x, y) == 0) continue;
                    uint64_t rank = (uint64_t)y * Rp + (uint64_t)(x / 3);
                    uint32_t u = site_u(&cache, seed, stream, (uint32_t)s,
                                        (uint32_t)slot, rank);
                    uint32_t t = t_site ? t_site[i] : t_scalar;
                    dec[i] = (u < t) ? 1 : 0;
                }
            or_lozenge_apply_pass(st, W, H, pass, dec);
        }
        if (hashes) hashes[s - sweep0] = or_state_hash(st, (uint64_t)3 * W * H);
    }
    free(dec);
    return 0;
}

/* q^volume weights: adding a cube multiplies the weight by q, so the       */
/* heat-bath add probability is q/(1+q); t_add = floor(2^32 q/(1+q)),      */
/* t_rem = 2^32 - t_add.                                                    */
OR_EXPORT int or_lozenge_thresholds(double q, uint32_t* t_add, uint32_t* t_rem)
{
    uint32_t ta = prob_to_threshold(q / (1.0 + q));
    if (ta == 0) return -1;
    *t_add = ta;
    *t_rem = (uint32_t)(((uint64_t)1 << 32) - (uint64_t)ta);
    return 0;
}

/* Triangles: up (x,y),(x+1,y),(x+1,y+1) with edges E1(x,y), E2(x+1,y),    */
/* E3(x,y); down (x,y),(x+1,y+1),(x,y+1) with edges E3(x,y), E2(x,y),      */
/* E1(x,y+1).  A lozenge covers the two triangles at its crossed edge.     */
static int tri_up(const uint8_t* st, int W, int H, int x, int y)
{
    return lget(st, W, H, 0, x, y) + lget(st, W, H, 1, x + 1, y) + lget(st, W, H, 2, x, y);
}
static int tri_dn(const uint8_t* st, int W, int H, int x, int y)
{
    return lget(st, W, H, 2, x, y) + lget(st, W, H, 1, x, y) + lget(st, W, H, 0, x, y + 1);
}

/* Validity: every triangle covered at most once; if masks are given (up    */
/* and down triangles, [H][W]), the covered set must equal them.           */
OR_EXPORT int64_t or_lozenge_check(const uint8_t* st, int W, int H,
                                   const uint8_t* up_mask, const uint8_t* dn_mask)
{
    int64_t bad = 0;
    for (int y = -1; y < H; ++y)
        for (int x = -1; x < W; ++x) {
            int cu = tri_up(st, W, H, x, y), cd = tri_dn(st, W, H, x, y);
            int in = x >= 0 && y >= 0;
            int wu = (up_mask && in) ? up_mask[(size_t)y * W + x] : (cu > 0);
            int wd = (dn_mask && in) ? dn_mask[(size_t)y * W + x] : (cd > 0);
            if (cu > 1 || cd > 1 || cu != wu || cd != wd) ++bad;
        }
    return bad;
}

/* Lozenge height: lift the tiling to the stepped surface of cubes and     */
/* take h = the k-coordinate of the lifted vertex (a lattice point         */
/* (x+k, y+k, k) up to the box offset).  An uncrossed edge is a cube edge: */
/* E1, E2 steps keep k, an E3 step is -e3 (k-1).  A crossed edge is the     */
/* short diagonal of a face: E1, E2 steps lower k by one, an E3 step keeps */
/* it.  Adding a cube at v raises h(v) by one.  h = 0 at the first domain  */
/* vertex in (y, x) order.                                                  */
OR_EXPORT int64_t or_lozenge_height(const uint8_t* st, int W, int H, int32_t* h)
{
    size_t nv = (size_t)W * H;
    int* queue = (int*)malloc(sizeof(int) * nv);
    if (!queue) return -1;
    for (size_t i = 0; i < nv; ++i) h[i] = HNONE;
#define TU(x, y) (tri_up(st, W, H, (x), (y)) == 1)
#define TD(x, y) (tri_dn(st, W, H, (x), (y)) == 1)
    /* a vertex is in the domain iff one of its six triangles is covered */
    int start = -1;
    for (int y = 0; y < H && start < 0; ++y)
        for (int x = 0; x < W && start < 0; ++x)
            if (TU(x, y) || TD(x, y) || TU(x - 1, y) || TD(x - 1, y - 1) ||
                TU(x - 1, y - 1) || TD(x, y - 1))
                start = y * W + x;
    if (start < 0) { free(queue); return 0; }
    int64_t bad = 0;
    size_t qh = 0, qt = 0;
    h[start] = 0; queue[qt++] = start;
    while (qh < qt) {
        int v = queue[qh++];
        int x = v % W, y = v / W;
        for (int d = 0; d < 6; ++d) {
            int nx, ny, dom, dh;
            switch (d) {
            case 0: /* +E1: edge E1(x,y) between up(x,y) and down(x,y-1) */
                nx = x + 1; ny = y; dom = TU(x, y) || TD(x, y - 1);
                dh = -lget(st, W, H, 0, x, y); break;
            case 1: /* -E1 */
                nx = x - 1; ny = y; dom = TU(x - 1, y) || TD(x - 1, y - 1);
                dh = +lget(st, W, H, 0, x - 1, y); break;
            case 2: /* +E2: edge E2(x,y) between down(x,y) and up(x-1,y) */
                nx = x; ny = y + 1; dom = TD(x, y) || TU(x - 1, y);
                dh = -lget(st, W, H, 1, x, y); break;
            case 3: /* -E2 */
                nx = x; ny = y - 1; dom = TD(x, y - 1) || TU(x - 1, y - 1);
                dh = +lget(st, W, H, 1, x, y - 1); break;
            case 4: /* +E3: edge E3(x,y) between up(x,y) and down(x,y) */
                nx = x + 1; ny = y + 1; dom = TU(x, y) || TD(x, y);
                dh = -1 + lget(st, W, H, 2, x, y); break;
            default: /* -E3 */
                nx = x - 1; ny = y - 1; dom = TU(x - 1, y - 1) || TD(x - 1, y - 1);
                dh = 1 - lget(st, W, H, 2, x - 1, y - 1); break;
            }
            if (!dom || nx < 0 || ny < 0 || nx >= W || ny >= H) continue;
            int32_t nh = h[v] + dh;
            int nv_ = ny * W + nx;
            if (h[nv_] == HNONE) { h[nv_] = nh; queue[qt++] = nv_; }
            else if (h[nv_] != nh) ++bad;
        }
    }
#undef TU
#undef TD
    free(queue);
    return bad;
}

/* ======================================================================== */
/* Six-vertex model (Sec. 1.2.4, Fig. 5, Fig. 6)                            */
/* ======================================================================== */
#define SH(st, B, X, Y) (st)[(size_t)(Y) * (B) + (X)]
#define SV(st, B, X, Y) (st)[(size_t)(B) * (B) + (size_t)(Y) * (B) + (X)]
static int sget_h(const uint8_t* st, int B, int X, int Y)
{
    if (X < 0 || Y < 0 || X >= B || Y >= B) return 0;
    return SH(st, B, X, Y);
}
static int sget_v(const uint8_t* st, int B, int X, int Y)
{
    if (X < 0 || Y < 0 || X >= B || Y >= B) return 0;
    return SV(st, B, X, Y);
}

/* Domain-wall boundary: paths enter through all N bottom external edges   */
/* and leave through all N left ones.  Start: path k (column k+1) goes up  */
/* to row k+1 and turns left (the identity alternating-sign matrix).       */
OR_EXPORT int or_sixv_dwbc_init(int N, uint8_t* st)
{
    int B = N + 2;
    memset(st, 0, (size_t)2 * B * B);
    for (int k = 0; k < N; ++k) {
        for (int Y = 0; Y <= k; ++Y) SV(st, B, k + 1, Y) = 1;
        for (int X = 0; X <= k; ++X) SH(st, B, X, k + 1) = 1;
    }
    return 0;
}

/* Vertex type at model vertex (X,Y) from its four edges (Fig. 5A):        */
/* L = Hz(X-1,Y), R = Hz(X,Y), D = Vt(X,Y-1), U = Vt(X,Y).  Paths enter by */
/* D or R and leave by U or L.  Returns 0..5 for a1,a2,b1,b2,c1,c2, or -1  */
/* if the ice rule fails.                                                   */
static int sixv_type(int L, int R, int D, int U)
{
    if (!L && !R && !D && !U) return 0;          /* a1: empty */
    if (L && R && D && U) return 1;              /* a2: full */
    if (L && R && !D && !U) return 2;            /* b1: horizontal through */
    if (!L && !R && D && U) return 3;            /* b2: vertical through */
    if (L && D && !R && !U) return 4;            /* c1: in below, out left */
    if (R && U && !L && !D) return 5;            /* c2: in right, out above */
    return -1;
}

OR_EXPORT int or_sixv_vertex_type(const uint8_t* st, int N, int X, int Y)
{
    int B = N + 2;
    return sixv_type(sget_h(st, B, X - 1, Y), sget_h(st, B, X, Y),
                     sget_v(st, B, X, Y - 1), sget_v(st, B, X, Y));
}

/* Number of model vertices violating the ice rule plus external edges     */
/* that differ from the domain-wall boundary.                               */
OR_EXPORT int64_t or_sixv_check_dwbc(const uint8_t* st, int N)
{
    int B = N + 2;
    int64_t bad = 0;
    for (int Y = 1; Y <= N; ++Y)
        for (int X = 1; X <= N; ++X)
            if (or_sixv_vertex_type(st, N, X, Y) < 0) ++bad;
    for (int k = 1; k <= N; ++k) {
        if (SH(st, B, 0, k) != 1) ++bad;   /* left: occupied */
        if (SV(st, B, k, 0) != 1) ++bad;   /* bottom: occupied */
        if (SH(st, B, N, k) != 0) ++bad;   /* right: empty */
        if (SV(st, B, k, N) != 0) ++bad;   /* top: empty */
    }
    return bad;
}

/* Face (X,Y) has lower-left vertex (X,Y) and edges B = Hz(X,Y),           */
/* T = Hz(X,Y+1), L = Vt(X,Y), R = Vt(X+1,Y).  The c-flip (Fig. 5C) swaps   */
/* a path turning through R,T (state A) with one through B,L (state B,      */
/* which is UP: the face height is two larger).  Interior faces only.      */
static int sixv_face_state(const uint8_t* st, int B, int X, int Y)
{
    int b = sget_h(st, B, X, Y), t = sget_h(st, B, X, Y + 1);
    int l = sget_v(st, B, X, Y), r = sget_v(st, B, X + 1, Y);
    if (b && l && !r && !t) return 2;
    if (r && t && !b && !l) return 1;
    return 0;
}

static void sixv_face_set(uint8_t* st, int B, int X, int Y, int up)
{
    SH(st, B, X, Y) = (uint8_t)up;
    SV(st, B, X, Y) = (uint8_t)up;
    SH(st, B, X, Y + 1) = (uint8_t)!up;
    SV(st, B, X + 1, Y) = (uint8_t)!up;
}

/* Four colour classes by the parities of the face coordinates (Sec.      */
/* 1.2.4), visited in the order (0,0), (1,1), (1,0), (0,1).                */
static const int SIXV_PX[4] = {0, 1, 1, 0};
static const int SIXV_PY[4] = {0, 1, 0, 1};

static int sixv_in_class(int N, int X, int Y, int pass)
{
    if (X < 1 || Y < 1 || X > N - 1 || Y > N - 1) return 0;
    return (X & 1) == SIXV_PX[pass] && (Y & 1) == SIXV_PY[pass];
}

OR_EXPORT void or_sixv_site_states(const uint8_t* st, int N, int pass, uint8_t* out)
{
    int B = N + 2;
    for (int Y = 0; Y < B; ++Y)
        for (int X = 0; X < B; ++X)
            out[(size_t)Y * B + X] = sixv_in_class(N, X, Y, pass)
                                         ? (uint8_t)sixv_face_state(st, B, X, Y)
                                         : 0;
}

OR_EXPORT void or_sixv_apply_pass(uint8_t* st, int N, int pass, const uint8_t* dec)
{
    int B = N + 2;
    for (int Y = 1; Y <= N - 1; ++Y)
        for (int X = 1; X <= N - 1; ++X) {
            if (!sixv_in_class(N, X, Y, pass)) continue;
            if (sixv_face_state(st, B, X, Y) == 0) continue;
            sixv_face_set(st, B, X, Y, dec[(size_t)Y * B + X] ? 1 : 0);
        }
}

/* The four corner vertices of a face each keep two external edges; the    */
/* flip leaves those alone.  Index of the threshold table: bit 0 = Vt(X,Y+1) */
/* (above the top-left corner), bit 1 = Hz(X+1,Y+1) (right of top-right),  */
/* bit 2 = Hz(X+1,Y) (right of bottom-right), bit 3 = Hz(X-1,Y) (left of   */
/* bottom-left).                                                            */
static int sixv_index(const uint8_t* st, int B, int X, int Y)
{
    return sget_v(st, B, X, Y + 1) | (sget_h(st, B, X + 1, Y + 1) << 1) |
           (sget_h(st, B, X + 1, Y) << 2) | (sget_h(st, B, X - 1, Y) << 3);
}

OR_EXPORT int or_sixv_sweeps(uint8_t* st, int N, const uint32_t t16[16],
                             uint64_t seed, uint32_t stream, uint64_t sweep0,
                             uint64_t nsweeps, uint64_t* hashes, int random_order)
{
    int B = N + 2;
    uint64_t Rp = round_up_128((uint64_t)(B + 1) / 2);
    uint8_t* dec = (uint8_t*)calloc((size_t)B * B, 1);
    if (!dec) return -1;
    u_cache cache; cache.valid = 0;
    for (uint64_t s = sweep0; s < sweep0 + nsweeps; ++s) {
        for (int slot = 0; slot < 4; ++slot) {
            const int pass = random_order ? or_slot_colour(seed, stream, (uint32_t)s, slot, 4) : slot;
            for (int Y = 0; Y < B; ++Y)
                for (int X = 0; X < B; ++X) {
                    size_t i = (size_t)Y * B + X;
                    dec[i] = 0;
                    if (!sixv_in_class(N, X, Y, pass)) continue;
                    if (sixv_face_state(st, B, X, Y) == 0) continue;
                    uint64_t rank = (uint64_t)(Y >> 1) * Rp + (uint64_t)(X >> 1);
                    uint32_t u = site_u(&cache, seed, stream, (uint32_t)s,
                                        (uint32_t)slot, rank);
                    dec[i] = (u < t16[sixv_index(st, B, X, Y)]) ? 1 : 0;
                }
            or_sixv_apply_pass(st, N, pass, dec);
        }
        if (hashes) hashes[s - sweep0] = or_state_hash(st, (uint64_t)2 * B * B);
    }
    free(dec);
    return 0;
}

/* Weight of a configuration: product over model vertices of the weight of */
/* its type (Sec. 1.2.4); w6 = (a1, a2, b1, b2, c1, c2).  Returns -1 if a  */
/* vertex breaks the ice rule.                                              */
OR_EXPORT double or_sixv_weight(const uint8_t* st, int N, const double w6[6])
{
    double prod = 1.0;
    for (int Y = 1; Y <= N; ++Y)
        for (int X = 1; X <= N; ++X) {
            int t = or_sixv_vertex_type(st, N, X, Y);
            if (t < 0) return -1.0;
            prod *= w6[t];
        }
    return prod;
}

/* Heat-bath table.  For each index the two local pictures (A and B) are   */
/* built explicitly on a 4x4 patch of edges around one face, the remaining  */
/* external edge of each corner is fixed by the ice rule, each corner is    */
/* classified, and t = floor(2^32 * W_B / (W_A + W_B)) with W the product */
/* of the four corner weights taken in the order TL, TR, BR, BL.           */
OR_EXPORT int or_sixv_thresholds(const double w6[6], uint32_t t16[16])
{
    for (int idx = 0; idx < 16; ++idx) {
        int tl = idx & 1, tr = (idx >> 1) & 1, br = (idx >> 2) & 1, bl = (idx >> 3) & 1;
        double wgt[2];
        for (int s = 0; s < 2; ++s) {
            int up = s;                 /* s = 0: state A, s = 1: state B */
            int fb = up, fl = up, fr = !up, ft = !up;   /* face edges */
            /* corners: BL (X,Y): L=bl (ext), R=fb, U=fl, D=? ; ice: L+U = D+R */
            int bl_D = bl + fl - fb; if (bl_D < 0 || bl_D > 1) return -1;
            int tBL = sixv_type(bl, fb, bl_D, fl);
            /* BR (X+1,Y): L=fb, R=br (ext), U=fr, D=? */
            int br_D = fb + fr - br; if (br_D < 0 || br_D > 1) return -1;
            int tBR = sixv_type(fb, br, br_D, fr);
            /* TL (X,Y+1): R=ft, D=fl, U=tl (ext), L=? */
            int tl_L = fl + ft - tl; if (tl_L < 0 || tl_L > 1) return -1;
            int tTL = sixv_type(tl_L, ft, fl, tl);
            /* TR (X+1,Y+1): L=ft, D=fr, R=tr (ext), U=? */
            int tr_U = fr + tr - ft; if (tr_U < 0 || tr_U > 1) return -1;
            int tTR = sixv_type(ft, tr, fr, tr_U);
            if (tBL < 0 || tBR < 0 || tTL < 0 || tTR < 0) return -1;
            wgt[s] = w6[tTL] * w6[tTR] * w6[tBR] * w6[tBL];
        }
        t16[idx] = prob_to_threshold(wgt[1] / (wgt[0] + wgt[1]));
    }
    return 0;
}

/* Six-vertex height on faces (Fig. 6): faces with lower-left vertex       */
/* (X,Y), 0 <= X,Y <= N, including the outer ring between external edges;  */
/* h = 0 at face (0,0); a step up across Hz(X,Y+1) adds +1 if occupied     */
/* and -1 if not; a step right across Vt(X+1,Y) likewise.  Output          */
/* [(N+1)][(N+1)], row-major in Y.  Returns inconsistencies.                */
OR_EXPORT int64_t or_sixv_height(const uint8_t* st, int N, int32_t* h)
{
    int B = N + 2, F = N + 1;
    int64_t bad = 0;
    /* first column by steps up, then every row by steps right, then check */
    h[0] = 0;
    for (int Y = 1; Y < F; ++Y)
        h[(size_t)Y * F] = h[(size_t)(Y - 1) * F] + (sget_h(st, B, 0, Y) ? 1 : -1);
    for (int Y = 0; Y < F; ++Y)
        for (int X = 1; X < F; ++X)
            h[(size_t)Y * F + X] = h[(size_t)Y * F + X - 1] + (sget_v(st, B, X, Y) ? 1 : -1);
    for (int Y = 1; Y < F; ++Y)
        for (int X = 0; X < F; ++X)
            if (h[(size_t)Y * F + X] != h[(size_t)(Y - 1) * F + X] + (sget_h(st, B, X, Y) ? 1 : -1))
                ++bad;
    return bad;
}

/* ======================================================================== */
/* Observables shared by all lattices                                        */
/* ======================================================================== */
/* Edge occupancy counters: counts[i] += st[i] for every canonical bit.    */
OR_EXPORT void or_accumulate(const uint8_t* st, uint64_t nbits, uint32_t* counts)
{
    for (uint64_t i = 0; i < nbits; ++i) counts[i] += st[i];
}
