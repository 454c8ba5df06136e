/*
 * tiling.h -- C-ABI of the GB300 sampler for random tilings by
 * colour-class-parallel heat-bath Glauber dynamics (Keating & Sridhar,
 * "Random Tilings with the GPU").
 *
 * The calls follow the paper's statement of the problem: a simply-connected
 * lattice domain (Sec. 1.1), an initial tiling (Sec. 1.1, Thurston), a random
 * walk of k sweeps driven by a seed (Sec. 2.2, host function RandomWalk) at
 * given edge / volume / vertex weights (Sec. 1.1.1, Sec. 1.2.1, Sec. 1.2.4),
 * and reading back the tiling, its height function (Sec. 1.1, Fig. 2; Fig. 6)
 * and observables.
 *
 * Conventions
 *  - Every call returns an int status: TL_OK (0) or a TL_E* code; nothing is
 *    thrown across the boundary.  tl_last_error() gives a thread-local
 *    message for the last failure on the calling thread.
 *  - The library owns the device memory of contexts, chains and batches and
 *    frees it in the matching *_destroy call.  Callers own every buffer they
 *    pass in.  A pointer argument documented as "host or device" may point to
 *    either; device pointers must belong to the context's GPU.
 *  - `stream` arguments are a cudaStream_t (NULL = legacy default stream).
 *    Calls that take a stream only enqueue work unless a host buffer is
 *    involved, in which case they synchronise that stream before returning.
 *  - A chain is not thread-safe; distinct chains may be driven from distinct
 *    threads.  Domains are immutable after creation and may be shared.
 *  - There is no CPU fallback: without a usable GPU every call that needs one
 *    returns TL_ECUDA.
 *
 * Canonical state (the interchange layout used by tl_read_state and
 * tl_chain_create): one uint8 (0 or 1) per lattice edge, [plane][y][x] over
 * the domain's vertex box of width W and height H (tl_domain_get_info).
 *  - Domino (Sec. 1.1, Sec. 2.2): plane 0 = edge (x,y)-(x+1,y), plane 1 =
 *    edge (x,y)-(x,y+1); 1 = a domino crosses the edge.  This stores each of
 *    the paper's redundant 4-bit tilestate bits once.
 *  - Lozenge (Sec. 1.2.1): axial triangular lattice, neighbours +-(1,0),
 *    +-(0,1), +-(1,1); planes 0,1,2 = edges to (x+1,y), (x,y+1), (x+1,y+1);
 *    1 = the edge is the short diagonal of a lozenge.
 *  - Six-vertex (Sec. 1.2.4): W = H = N+2 with the N x N model vertices at
 *    1..N; plane 0 = edge east of (X,Y), plane 1 = edge north of (X,Y);
 *    1 = occupied.  External half-edges are plane 0 at X = 0 and X = N and
 *    plane 1 at Y = 0 and Y = N.
 *
 * Randomness: a flippable site goes UP iff u < t, where t is its heat-bath
 * threshold and u a 32-bit uniform whose bit (31-k) is bit (rank & 31) of
 * output word ((rank >> 5) & 3) of Philox4x32-10 (Salmon et al., SC'11)
 * with key (seed & 0xffffffff, seed >> 32) and counter
 * (rank >> 7, sweep, (k << 16) | pass, stream_id).  rank = r * Rp + j where
 * (r, j) = (y, x >> 1) for dominoes, (y, x / 3) for lozenges and
 * (Y >> 1, X >> 1) for six-vertex faces, and Rp is the number of j values
 * per row rounded up to a multiple of 128.  `sweep` is the absolute sweep
 * index since chain creation.  Results therefore do not depend on launch
 * shape, batching or serving.  UP means: two vertical dominoes (tilestate
 * 12, Sec. 2.2), a cube added (Sec. 1.2.1), or the six-vertex face path
 * through its bottom and left edges (Fig. 5C).
 *
 * Passes: a sweep visits the colour classes in a fixed order -- dominoes
 * (x+y) mod 2 = 0, 1 (Sec. 1.1.3); lozenges (x+y) mod 3 = 0, 1, 2 (Sec.
 * 1.2.1); six-vertex faces by (X mod 2, Y mod 2) = (0,0), (1,1), (1,0),
 * (0,1) (Sec. 1.2.4).  All sites of a class move at once (Eq. 1.1).
 */
#ifndef TILING_H
#define TILING_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    TL_OK = 0,
    TL_EINVAL = 1,        /* bad argument, size or state */
    TL_ENOTSIMPLY = 2,    /* domain boundary is not a simple closed path */
    TL_ENOTTILEABLE = 3,  /* domain has no tiling */
    TL_ENOMEM = 4,        /* host or device allocation failed */
    TL_EBUDGET = 5,       /* request exceeds a memory budget */
    TL_ECUDA = 6,         /* CUDA runtime error (message has details) */
    TL_ETIMEOUT = 7,      /* a bounded device-side wait gave up */
    TL_EBUSY = 8,         /* resource in use */
    TL_EUNSUPPORTED = 9   /* valid request the library does not implement */
};

typedef enum { TL_DOMINO = 0, TL_LOZENGE = 1, TL_SIXV = 2 } tl_lattice;

typedef struct tl_ctx tl_ctx;
typedef struct tl_domain tl_domain;
typedef struct tl_chain tl_chain;

/* Thread-local message describing the last failing call on this thread. */
const char* tl_last_error(void);

/* Library version string. */
const char* tl_version(void);

/* ------------------------------------------------------------------------
 * Context: one per GPU.  cuda_device is the CUDA ordinal.  The context
 * records the device's SM count and shared-memory limits used by the
 * launch planner.  tl_ctx_destroy releases the caller's handle; chains and
 * batches created on the context hold it too, and it is freed when the last
 * of them is destroyed, in any order.  Errors: TL_EINVAL (bad ordinal),
 * TL_ECUDA.
 * ---------------------------------------------------------------------- */
int tl_ctx_create(int cuda_device, tl_ctx** out);
void tl_ctx_destroy(tl_ctx* ctx);

/* Context options.  max_sms: use at most this many SMs for the resident
 * kernels' stripes and the batched kernel's grid (0 = all), leaving the rest
 * of the GPU to other work; results never depend on it.  Errors as
 * tl_ctx_create, and TL_EINVAL for a negative field. */
typedef struct {
    int max_sms;
} tl_ctx_opts;
int tl_ctx_create_opts(int cuda_device, const tl_ctx_opts* opts, tl_ctx** out);

/* ------------------------------------------------------------------------
 * Domains (Sec. 1.1: a simply-connected union of lattice faces; Sec. 1.2.1
 * lozenge hexagon; Sec. 1.2.4 six-vertex box with fixed boundary).
 *  tl_domain_aztec:   Aztec diamond of order n >= 1 (faces with centres
 *                     |cx-n| + |cy-n| <= n), box (2n+1)^2, start: every row
 *                     of faces tiled by horizontal dominoes.
 *  tl_domain_rect:    w x h faces, box (w+1) x (h+1); start all-horizontal
 *                     (w even) or all-vertical (h even); TL_ENOTTILEABLE if
 *                     w*h is odd.
 *  tl_domain_hexagon: hexagon with sides a, b, c (an a x b x c box of cubes
 *                     seen along (1,1,1)); box (a+c+1) x (b+c+1); start: the
 *                     empty box (minimal height).
 *  tl_domain_dwbc:    six-vertex N x N with domain-wall boundary (all bottom
 *                     and left external edges occupied, top and right empty);
 *                     start: the identity permutation (path k enters column k
 *                     and turns left at row k).
 * Sizes: every box side must be <= 65536 and the box <= 2^31 vertices;
 * otherwise TL_EINVAL.  Domains live on the host and are freed with
 * tl_domain_destroy.
 * ---------------------------------------------------------------------- */
int tl_domain_aztec(int n, tl_domain** out);
int tl_domain_rect(int w, int h, tl_domain** out);
int tl_domain_hexagon(int a, int b, int c, tl_domain** out);
int tl_domain_dwbc(int N, tl_domain** out);
void tl_domain_destroy(tl_domain* d);

typedef struct {
    int lattice;            /* tl_lattice */
    int width, height;      /* vertex box W x H */
    int planes;             /* canonical planes: 2 or 3 */
    int passes;             /* colour classes per sweep: 2, 3 or 4 */
    uint64_t sites;         /* flip attempts per sweep (interior sites) */
    uint64_t edges;         /* non-redundant state bits (dual edges for
                               dominoes/lozenges, lattice edges for 6V) */
    uint64_t canon_bytes;   /* planes * W * H */
    uint64_t packed_bytes;  /* device bytes of one chain's packed state */
    uint64_t site_box;      /* W * H: entries of a per-site threshold array */
    uint64_t height_count;  /* entries of tl_read_height output */
    int height_width;       /* height grid width (W, or N+1 for 6V) */
    int height_height;
} tl_domain_info;

int tl_domain_get_info(const tl_domain* d, tl_domain_info* out);

/* Copy the domain's canonical starting tiling into `canon` (host, cap >=
 * canon_bytes). */
int tl_domain_initial_state(const tl_domain* d, uint8_t* canon, size_t cap);

/* Extreme configurations (Sec. 1.1: the maximal and minimal tilings T_max
 * and T_min of the distributive lattice of tilings, found by Thurston's
 * algorithm in time proportional to the domain size).  TL_EXTREME_TOP has
 * the largest height function (dominoes: Fig. 2 with h = 0 at the first
 * domain vertex; lozenges: every rotatable site UP, a full box for a
 * hexagon; six-vertex: every face in state B, the anti-diagonal permutation
 * for the domain wall), TL_EXTREME_BOTTOM the smallest (lozenges and
 * six-vertex: every rotatable site DOWN, the built-in starting
 * configurations).  For dominoes a rotation raises the height at sites of
 * one colour and lowers it at the other, so both mix UP and DOWN blocks;
 * the all-horizontal start of the Aztec diamond of order n is T_max for
 * even n and T_min for odd n.  These are the two chains started by coupling
 * from the past (Sec. 1.1.4).  `canon` is host memory, cap >= canon_bytes.
 * Errors: TL_EINVAL. */
#define TL_EXTREME_BOTTOM 0
#define TL_EXTREME_TOP 1
int tl_domain_extreme_state(const tl_domain* d, int which, uint8_t* canon, size_t cap);

/* Domain enclosed by a closed lattice path (Sec. 1.1: a simply-connected
 * union of faces; tileability and a starting tiling by Thurston's
 * algorithm).  The path starts at a lattice point and takes `nsteps` unit
 * steps `steps[i]`:
 *   TL_DOMINO: 0 = +x, 1 = +y, 2 = -x, 3 = -y (square lattice);
 *   TL_LOZENGE: 0 = +x, 1 = +y, 2 = +x+y, 3 = -x, 4 = -y, 5 = -x-y
 *   (triangular lattice in the axial coordinates of the canonical layout).
 * It must return to its start and visit no other point twice; either
 * orientation.  The domain is translated so that the path's lowest x and y
 * are 0; its starting configuration is TL_EXTREME_BOTTOM.  Errors:
 * TL_EINVAL (bad lattice or step, path not closed, too large),
 * TL_ENOTSIMPLY (path crosses itself), TL_ENOTTILEABLE (no tiling). */
int tl_domain_from_boundary(int lattice, const int8_t* steps, size_t nsteps, tl_domain** out);

/* ------------------------------------------------------------------------
 * Heat-bath thresholds, computed once on the host in FP64.  In each case
 * t = floor(P(UP) * 2^32), clamped to [0, 2^32 - 1], with P(UP) evaluated
 * exactly in the order written below.
 *
 * Domino edge weights (Sec. 1.1.1): `w` is laid out like the canonical
 * state ([2][H][W] doubles, weight of the dual edge crossing each primal
 * edge; n_w = 2*W*H).  For each vertex (x,y): up = wE*wW, down = wN*wS with
 * wE = w[0][y][x], wW = w[0][y][x-1], wN = w[1][y][x], wS = w[1][y-1][x]
 * (1.0 outside the box), P = up / (up + down).  Output t[y][x] for every box
 * vertex (n_t = W*H).  Errors: TL_EINVAL on size mismatch, non-positive or
 * non-finite weights.
 * ---------------------------------------------------------------------- */
int tl_thresholds_domino_edge_weights(const tl_domain* d, const double* w, size_t n_w,
                                      uint32_t* t, size_t n_t);

/* Volume weights (Sec. 1.1.1: W(T) = prod over vertices of q_v^{h_T(v)};
 * for lozenges the height is the cube-stack height, so q_v weighs each cube
 * stacked at v).  `q` is [H][W] doubles, one per box vertex (n_q = W*H).
 * A domino rotation at (x,y) changes only h(x,y), by 4; UP raises it when
 * x + y is even and lowers it when odd (Fig. 2 with h = 0 at the first
 * domain vertex), so with q4 = (q*q)*(q*q): P = q4 / (1 + q4) for x + y
 * even and 1 / (1 + q4) for x + y odd.  Lozenges: P(add) = q / (1 + q).
 * Output t[y][x] (n_t = W*H) for use as per-site thresholds.  Errors:
 * TL_EINVAL (six-vertex domain, size mismatch, q outside [1e-75, 1e75],
 * where q^4 would leave the normal doubles). */
int tl_thresholds_volume(const tl_domain* d, const double* q, size_t n_q, uint32_t* t, size_t n_t);

/* Generated log-normal weights (weight = exp(sigma Z), Z standard normal),
 * drawn on the device from Philox4x32-10 keyed by `seed` and the canonical
 * index of each edge (dominoes: dual-edge weights, thresholds as in
 * tl_thresholds_domino_edge_weights) or vertex (lozenges: volume weight q_v,
 * P(add) = q_v / (1 + q_v)).  Writes t[H][W] into device memory `t_dev`
 * (n_t >= W*H) on `stream`; the FP64 threshold arithmetic uses correctly
 * rounded operations in the order given above.  For workloads whose weights
 * are random, such as served sampling jobs.  Six-vertex: TL_EINVAL. */
int tl_thresholds_lognormal_device(const tl_domain* d, double sigma, uint64_t seed, uint32_t* t_dev, size_t n_t,
                                   void* stream);

/* Lozenge q^volume (Sec. 1.1.1 volume weights on the cube picture, Sec.
 * 1.2.1): P(add a cube) = q / (1 + q); t_add as above, t_rem = 2^32 - t_add.
 * A flippable site ends with the cube present iff u < t_add.  TL_EINVAL if q
 * is not positive and finite or t_add would be 0. */
int tl_thresholds_lozenge_q(double q, uint32_t* t_add, uint32_t* t_rem);

/* Six-vertex vertex weights (Sec. 1.2.4, Fig. 5A) w6 = (a1, a2, b1, b2, c1,
 * c2).  t16[idx] for the face flip (Fig. 5C) given the four external corner
 * bits idx = Vt(X,Y+1) | Hz(X+1,Y+1) << 1 | Hz(X+1,Y) << 2 | Hz(X-1,Y) << 3:
 * W_A and W_B are the products of the four corner-vertex weights in the order
 * top-left, top-right, bottom-right, bottom-left for the face's two states
 * (A = path through right and top edges, B = through bottom and left = UP),
 * and P = W_B / (W_A + W_B). */
int tl_thresholds_6v(const double w6[6], uint32_t t16[16]);

/* ------------------------------------------------------------------------
 * Chains.
 * ---------------------------------------------------------------------- */
typedef enum {
    TL_T_SCALAR = 0,   /* one threshold for every site (domino, lozenge) */
    TL_T_SITE = 1,     /* per-site thresholds (domino, lozenge) */
    TL_T_TABLE16 = 2   /* six-vertex 16-entry table */
} tl_threshold_kind;

typedef struct {
    int kind;                 /* tl_threshold_kind */
    uint32_t scalar;          /* TL_T_SCALAR */
    const uint32_t* site;     /* TL_T_SITE: host or device array [H][W] (t per vertex) */
    uint32_t table16[16];     /* TL_T_TABLE16 */
} tl_thresholds;

/* Create a chain on `ctx` for domain `d`.  `canon_init` (host, canon_bytes)
 * is the starting tiling, or NULL for the domain's default start; it is
 * checked (every face / triangle covered once, or the ice rule and the
 * boundary for six-vertex) and TL_EINVAL is returned if it is not a valid
 * configuration of the domain.  `seed` keys the Philox generator,
 * `stream_id` separates independent chains.  The thresholds are copied.
 * The chain's sweep counter starts at 0.  Errors: TL_EINVAL, TL_ENOMEM,
 * TL_ECUDA. */
int tl_chain_create(tl_ctx* ctx, const tl_domain* d, const uint8_t* canon_init,
                    uint64_t seed, uint32_t stream_id, const tl_thresholds* th,
                    tl_chain** out);
void tl_chain_destroy(tl_chain* c);

/* Restore the chain to its creation state on `stream`: the starting
 * configuration (from a device-side copy taken at creation), sweep counter
 * 0, density sampling off.  Enqueues only. */
int tl_chain_reset(tl_chain* c, void* stream);

/* Absolute sweep index of the chain (number of sweeps run so far). */
uint64_t tl_chain_sweep(const tl_chain* c);

/* Pass order of the chain's sweeps.  TL_ORDER_FIXED (default) visits the
 * colour classes in their fixed order (dominoes 0, 1; lozenges 0, 1, 2;
 * six-vertex (0,0), (1,1), (1,0), (0,1)).  TL_ORDER_RANDOM follows
 * RandomWalk (Sec. 2.2), which picks the colour of every step at random:
 * slot i of sweep s updates colour floor(P w / 2^32), P the number of
 * colours and w word 0 of Philox4x32-10(key = seed, counter = (2^32 - 1, s,
 * 0xFFFF0000 | i, stream_id)), and the site draws of that slot use pass
 * field i.  Every pass preserves the Gibbs measure, so both orders sample
 * it.  Chains with the random order cannot join a batch (TL_EUNSUPPORTED
 * there).  Choosing TL_ORDER_RANDOM waits for the device once and allocates
 * the chain's buffer of slot colours (3.84 MB, enough for any launch), so
 * tl_run_sweeps still only enqueues.  Errors: TL_EINVAL, TL_ENOMEM,
 * TL_ECUDA. */
#define TL_ORDER_FIXED 0
#define TL_ORDER_RANDOM 1
int tl_chain_set_order(tl_chain* c, int order);

/* Accepted-flip counter (a chain metric): after tl_chain_count_flips(c, 1)
 * every site rotation that the chain's own sweeps perform (tl_run_sweeps,
 * tl_run_sweeps_hashed; a site that changes orientation in a pass counts
 * once) is added to a 64-bit device counter, which the call resets;
 * tl_chain_count_flips(c, 0) stops counting.  tl_chain_flips waits for the
 * device and reads the count.  Sweeps run inside a batch are not counted.
 * The ratio flips / (sites x sweeps) is the chain's acceptance rate.
 * Errors: TL_EINVAL, TL_ENOMEM, TL_ECUDA. */
int tl_chain_count_flips(tl_chain* c, int on);
int tl_chain_flips(tl_chain* c, uint64_t* out);

/* Set the absolute index of the next sweep (0 .. 2^32 - 1).  Random numbers
 * are keyed by this index, so seeking replays or skips randomness; coupling
 * from the past uses it to place runs at negative times.  Sweeps run after a
 * seek must stay below 2^32.  Errors: TL_EINVAL. */
int tl_chain_seek(tl_chain* c, uint64_t sweep);

/* Checkpoints (the position and inputs of RandomWalk, Sec. 2.2, carried
 * across processes).  tl_checkpoint waits for the device, then writes into
 * `out` a library-allocated byte string (free it with tl_blob_free) holding
 * the lattice and box, seed, stream id, next sweep index, pass order,
 * thresholds as given to tl_chain_create, the chain's starting tiling and
 * its current tiling; layout: a fixed header, then the two canonical states,
 * then the per-site thresholds (if any), in the host's byte order.  Density
 * counters and the launch plan are not saved.  tl_restore builds on `ctx` a
 * new chain with the same domain (the faces its starting tiling covers; the
 * six-vertex square from its size), inputs, state and sweep index, so that
 * running k sweeps on it gives exactly what the original would have.
 * Errors: TL_EINVAL (NULL, not a checkpoint, corrupt), TL_ENOMEM, TL_ECUDA. */
typedef struct {
    void* data;
    size_t size;
} tl_blob;
int tl_checkpoint(tl_chain* c, tl_blob* out);
int tl_restore(tl_ctx* ctx, const tl_blob* blob, tl_chain** out);
void tl_blob_free(tl_blob* b);

/* Exact uniform random tiling of the Aztec diamond of order n (1 <= n <=
 * 32767) by domino shuffling (the shuffling algorithms of Sec. 3; Elkies,
 * Kuperberg, Larsen and Propp), independent of the Markov chain: n growth
 * steps of destruction, sliding and creation, all on the device.  The draw
 * of the 2x2 block created with lower-left cell (x, y) (cells centred on the
 * diamond, x, y in [-n, n)) at order K is word 0 of Philox4x32-10(key =
 * seed, counter = ((y+n) << 16 | (x+n), K, 0xFFFE0000, stream_id)): two
 * horizontal dominoes if it is below 2^31, else two vertical ones.  Writes
 * the canonical state of tl_domain_aztec(n) to `canon` (host or device, cap
 * >= 2 (2n+1)^2).  Synchronous.  The context keeps the device buffers
 * (about 20 n^2 bytes) and one captured graph of the whole sample
 * for the last order used, until tl_ctx_destroy or a call with another
 * order; calls on one context are serialised.  Errors: TL_EINVAL,
 * TL_ENOMEM, TL_ECUDA. */
int tl_aztec_shuffle(tl_ctx* ctx, int n, uint64_t seed, uint32_t stream_id, uint8_t* canon, size_t cap,
                     void* stream);

/* Exact sample by coupling from the past (Sec. 1.1.4; Propp and Wilson).
 * Two chains start from TL_EXTREME_TOP and TL_EXTREME_BOTTOM with the same
 * seed and stream id and run the sweeps with absolute indices 2^32 - T ..
 * 2^32 - 1 (negative times -T .. -1), for T = t0, 2 t0, 4 t0, ...; the
 * heat-bath move is monotone for dominoes and lozenges (and for the
 * six-vertex model when a <= c and b <= c, Sec. 1.2.4), so once both chains
 * end in the same configuration every start would have, and that
 * configuration is an exact sample.  Coalescence is detected by equal state
 * hashes and confirmed by comparing the configurations.  The result goes to
 * `canon_out` (host or device, cap >= canon_bytes) and the T used to
 * *t_used.  Synchronous.  Errors: TL_EINVAL (t0 < 1, tmax < t0 or tmax >
 * 2^31), TL_EBUDGET (no coalescence within tmax sweeps), TL_ENOMEM,
 * TL_ECUDA, TL_ETIMEOUT. */
int tl_cftp(tl_ctx* ctx, const tl_domain* d, uint64_t seed, uint32_t stream_id, const tl_thresholds* th,
            uint64_t t0, uint64_t tmax, uint8_t* canon_out, size_t cap, uint64_t* t_used, void* stream);

/* Run k sweeps (the loop of RandomWalk, Sec. 2.2, with a fixed pass order)
 * on `stream`.  Enqueues only.  Density samples due inside the range (see
 * tl_density_begin) are taken at the right sweeps.  Errors: TL_EINVAL,
 * TL_ECUDA, TL_ETIMEOUT (a bounded device wait gave up; the chain's state is
 * then undefined). */
int tl_run_sweeps(tl_chain* c, uint64_t k, void* stream);

/* Run k sweeps one at a time and write the state hash after every sweep
 * into ring[0..k-1] (uint64, host or device).  Slower; for verification. */
int tl_run_sweeps_hashed(tl_chain* c, uint64_t k, uint64_t* ring, void* stream);

/* Canonical state of the chain into `canon` (host or device, cap >=
 * canon_bytes). */
int tl_read_state(tl_chain* c, uint8_t* canon, size_t cap, void* stream);

/* Replace the chain's state (host or device canonical buffer, n ==
 * canon_bytes).  The configuration is validated as in tl_chain_create (every
 * byte 0 or 1; every face covered once, or the six-vertex boundary and ice
 * rule), on the device: host bytes are first copied into the chain's
 * scratch.  TL_EINVAL names the first failure and leaves the chain's state
 * unchanged.  Returns once the check is done (the caller's buffer may then
 * be reused); the packing is enqueued on `stream`. */
int tl_write_state(tl_chain* c, const uint8_t* canon, size_t n, void* stream);

/* Order-independent state hash: sum mod 2^64 over set canonical bits i of
 * splitmix64(i) (Steele, Lea & Flood 2014; mix of x + 0x9e3779b97f4a7c15).
 * `out` is host or device. */
int tl_state_hash(tl_chain* c, uint64_t* out, void* stream);

/* Height function (Sec. 1.1 and Fig. 2 for dominoes: +-1 along uncrossed
 * edges with a black face on the left counting +1, -+3 across dominoes;
 * lozenges: the k-coordinate of the cube surface, raised by one per added
 * cube; six-vertex Fig. 6: face heights, +1 across occupied and -1 across
 * empty edges stepping up or right).  h = 0 at the first domain vertex in
 * (y, x) order (six-vertex: the bottom-left outer face).  Output int32
 * [height_height][height_width] (host or device); vertices off the domain
 * get INT32_MIN. */
int tl_read_height(tl_chain* c, int32_t* out, size_t cap, void* stream);

/* Height function without allocating anything (the paper has no
 * counterpart; it is an interface for callers that cannot call cudaMalloc
 * when they need the heights, e.g. code under a device-memory budget that
 * forbids new allocations, or a loop that must not pay the device-wide
 * synchronisation cudaMalloc / cudaFree can cause).  Same result as
 * tl_read_height, but `out` must be device memory of the chain's GPU
 * (TL_EINVAL otherwise), and the per-segment scratch that tl_read_height
 * keeps in chain-owned memory lives in one static device array of 65536 ints
 * (256 KiB) that every GPU using the library holds until the process exits.
 * A height segment is a maximal run of domain vertices in one row: one per
 * row for the Aztec diamond, rectangles, hexagons and the domain-wall square,
 * possibly several per row for non-convex domains from a boundary path;
 * domains with more than 65536 segments are rejected with TL_EINVAL.  The
 * array's device address is looked up by tl_ctx_create, once per device.
 * All calls on a device share the array and each rewrites the entries it
 * uses, so calls whose work overlaps on the GPU (different streams,
 * concurrently) race and must be serialised by the caller.  Enqueues on
 * `stream` only. */
int tl_read_height_noalloc(tl_chain* c, int32_t* out, size_t cap, void* stream);

/* Edge-occupancy sampling (the densities of Sec. 4's figures).  After this
 * call every sweep s with s >= burn_in and (s - burn_in) % stride == 0
 * that a later tl_run_sweeps completes (s counted after the sweep, 1-based)
 * adds the state to per-edge uint32 counters.  Resets the counters. */
int tl_density_begin(tl_chain* c, uint32_t stride, uint64_t burn_in);

/* Per-edge density = count / samples in FP64, canonical layout
 * [planes][H][W] (host or device doubles, cap >= canon_bytes entries).
 * *samples (host, may be NULL) receives the number of samples. */
int tl_read_density(tl_chain* c, double* out, size_t cap, uint64_t* samples, void* stream);

/* Domino only: per-face densities of the four domino types, [4][H-1][W-1]
 * doubles (host or device) in the order north, south, east, west.  A
 * horizontal domino is north iff its left square has the colour (x+y) mod 2
 * == kappa; a vertical one is west iff its bottom square has colour
 * (x+y) mod 2 != kappa; kappa = n mod 2 for the Aztec diamond of order n
 * (so the all-horizontal start is north in the upper half) and 0 otherwise. */
int tl_read_domino_nsew(tl_chain* c, double* out, size_t cap, void* stream);

/* Launch plan of a chain.  Every field 0 means "automatic".  Results never
 * depend on the plan: the random numbers are keyed by site and sweep.
 *  kernel:            1 one launch per pass over global memory; 2 the
 *                     shared-memory resident multi-sweep kernel (cooperative
 *                     launch; TL_EUNSUPPORTED if the domain does not fit it);
 *                     3 the register-resident multi-sweep kernel for
 *                     dominoes at t = 2^31 (every 128-site group of a row
 *                     pair held in one thread's registers; the automatic
 *                     choice for such chains when it fits, TL_EUNSUPPORTED
 *                     otherwise).
 *  sweeps_per_launch: cap on sweeps per resident launch.
 *  halo:              passes between boundary exchanges of the resident
 *                     kernels (1..64; even for kernel 3).
 *  threads:           threads per CTA of the resident kernel (512 or 1024).
 *  npre:              random bit planes generated ahead per group (1..16).
 * tl_chain_get_plan also fills the resolved values and ctas / smem_bytes. */
typedef struct {
    int kernel;
    int sweeps_per_launch;
    int halo;
    int threads;
    int npre;
    int ctas;            /* out: CTAs of the resident kernel (0 if not used) */
    int smem_bytes;      /* out: dynamic shared memory per CTA */
} tl_plan;

int tl_chain_set_plan(tl_chain* c, const tl_plan* plan);
int tl_chain_get_plan(tl_chain* c, tl_plan* plan);

/* Wait for the chain's work on `stream` and report a failure of the
 * resident kernel's bounded waits (TL_ETIMEOUT; the state is then
 * undefined and should be rewritten with tl_write_state or tl_chain_reset). */
int tl_chain_sync(tl_chain* c, void* stream);

/* Count of kernel launches the library made on this chain since creation
 * (all kinds).  For accounting in benchmarks. */
uint64_t tl_chain_launches(const tl_chain* c);

/* ------------------------------------------------------------------------
 * Batched chains (many independent samples of possibly different domains
 * and lattices advanced together; the multi-sample experiments of Sec. 4).
 * A batch references existing chains (it does not own them) and adds a
 * second device buffer per chain.  tl_batch_run advances every chain by k
 * sweeps: each launch runs R sweeps on every tile (a stripe of tile_rows
 * rows plus a halo of R * passes rows) of every chain, tiles taken largest
 * first from one work list; blocks of `graph_block` sweeps are replayed as a
 * CUDA graph when `stream` is not the legacy stream.  Every chain ends in
 * exactly the state, sweep count and hash it would reach with
 * tl_run_sweeps alone (random numbers are keyed by site, sweep and the
 * chain's own stream id).  While in a batch, chains must not sample
 * densities (TL_EINVAL at creation); they may still be read and run alone
 * between batch calls.
 * ---------------------------------------------------------------------- */
typedef struct tl_batch tl_batch;

/* Test hook for the failure path (no counterpart in the paper): raises the
 * status word that the bounded waits of the resident kernels (chain `c`, if
 * not NULL) and of the batched kernel (batch `b`, if not NULL) raise when they
 * give up.  Their next launches stop at their first wait point (the next
 * boundary exchange, the next tile) as if a wait had run out, so
 * tl_chain_sync / tl_batch_hashes report TL_ETIMEOUT, clear the word, and
 * leave the states undefined until tl_write_state or tl_chain_reset.
 * Nothing waits longer and no fault is raised.  TL_EUNSUPPORTED if the chain
 * runs on the per-pass kernel (it has no waits). */
int tl_debug_raise_status(tl_chain* c, tl_batch* b);

/* Bounds-checked build (no counterpart in the paper): libtiling_debug.so,
 * built with -DTL_DEBUG (`python paper_1804_07250_gb300/_build.py --debug`),
 * checks the computed indices of the kernels' shared-memory and global
 * accesses (the register and shared-memory resident kernels, the batched
 * kernel, the per-pass and read-back kernels, domino shuffling).  An index
 * outside its buffer is counted and the access skipped, so a wrong index
 * becomes a reported failure instead of a fault; results with no failure
 * are those of the normal build.
 *  tl_debug_build:    1 in the checked build, 0 in the normal one.
 *  tl_debug_checks:   waits for the device, then reports the failed checks
 *                     of every kernel file since the last clear: their count
 *                     (`failures`), and the id, index and bound of the first
 *                     (each pointer may be NULL); clears them if `clear`.
 *                     TL_EUNSUPPORTED in the normal build.
 *  tl_debug_selftest: runs one check of an index out of its range (index 5,
 *                     bound 3, id 999) whose access is skipped; a following
 *                     tl_debug_checks reports it.  TL_EUNSUPPORTED in the
 *                     normal build. */
int tl_debug_build(void);
int tl_debug_checks(int clear, uint64_t* failures, int* first_id, int64_t* index, int64_t* bound);
int tl_debug_selftest(void);

typedef struct {
    int tile_rows;          /* rows per tile (0 = keep) */
    int sweeps_per_launch;  /* R (0 = keep) */
    int graph_block;        /* sweeps per CUDA-graph block (0 = keep; default 100;
                               -1 = never capture graphs, e.g. while other threads
                               use the legacy stream) */
    int grid;               /* out: CTAs per launch */
    int smem_bytes;         /* out: dynamic shared memory per CTA */
    int ntiles;             /* out: tiles in the work list */
    int threads;            /* threads per tile, 256 or 128 (0 = keep; default
                               256): a thread takes every threads-th 128-face
                               group of a pass, so this sets the faces per
                               thread (128 threads: twice as many, with more
                               tiles resident per SM where shared memory
                               allows) */
} tl_batch_plan;

int tl_batch_create(tl_ctx* ctx, tl_chain* const* chains, size_t n, tl_batch** out);
void tl_batch_destroy(tl_batch* b);
/* Continuous batching: add a chain to / remove a chain from the batch
 * between runs (the work list is re-planned; removal waits for the device). */
int tl_batch_add(tl_batch* b, tl_chain* c);
int tl_batch_remove(tl_batch* b, tl_chain* c);
size_t tl_batch_size(const tl_batch* b);
int tl_batch_run(tl_batch* b, uint64_t k, void* stream);
/* The comparison point: the same kernel launched once per chain per R
 * sweeps (no batching, no graph). */
int tl_batch_run_per_chain(tl_batch* b, uint64_t k, void* stream);
/* State hash of every chain (uint64 out[n], host or device, n >= chains).
 * With a host `out` the call waits for the stream and reports TL_ETIMEOUT if
 * a batch launch gave up waiting for a tile's bulk copy (bounded at two
 * seconds; the chain states are then undefined). */
int tl_batch_hashes(tl_batch* b, uint64_t* out, size_t n, void* stream);
int tl_batch_set_plan(tl_batch* b, const tl_batch_plan* plan);
int tl_batch_get_plan(tl_batch* b, tl_batch_plan* plan);
/* Time every tile height in {32, 64, 128} x R in {1, 2, 4, 8} x threads per
 * tile in {256, 128} (the faces per thread) on the batch itself for
 * `trial_sweeps` sweeps (rounded up to a multiple of R), twice
 * each from the same states, and keep the plan with the fastest run; states
 * and sweep counters are restored afterwards.  The result is cached per
 * (lattices present, threshold kinds present, total rows rounded down to a
 * power of two, SM count): a later batch with the same key takes the cached
 * plan at once, without trials.  tl_autotune_cache_clear empties the cache. */
int tl_batch_autotune(tl_batch* b, uint64_t trial_sweeps, void* stream, tl_batch_plan* out);
void tl_autotune_cache_clear(void);
uint64_t tl_batch_launches(const tl_batch* b);

#ifdef __cplusplus
}
#endif

#endif /* TILING_H */
