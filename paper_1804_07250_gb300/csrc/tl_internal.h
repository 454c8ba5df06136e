// Internal declarations shared by the host runtime (tl_host.cpp) and the CUDA
// kernels (tl_kernels.cu).  Not part of the public C-ABI.
//
// Packed device layout of one chain ("rows"):
//   for every vertex row y of the box (plus one zero pad row below and one
//   above), P bit planes of K uint32 words each, plane = type * npar + res.
//   Bit j of a plane row holds the edge of type `type` at x = npar * j + res:
//     dominoes    npar 2, types {Hz, Vt}          (P = 4)
//     lozenges    npar 3, types {E1, E2, E3}      (P = 9)
//     six-vertex  npar 2, types {Hz, Vt}          (P = 4)
//   so every word holds 32 sites of one colour class of one row, and a
//   128-site group (4 words) is exactly one Philox4x32 output of the keying.
//   K = (j values per row rounded up to 128) / 32.  Rows are 16-byte
//   aligned; word (y, plane, k) lives at rows[((y + 1) * P + plane) * K + k].
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace tl {

enum Lattice : int { LAT_DOMINO = 0, LAT_LOZENGE = 1, LAT_SIXV = 2 };
enum ThrKind : int { THR_SCALAR = 0, THR_SITE = 1, THR_TABLE = 2 };

struct Geom {
    int lattice;
    int W, H;        // vertex box
    int N;           // six-vertex size (W = H = N + 2), else 0
    int npar;        // x residues per plane type
    int ntype;       // plane types
    int P;           // planes per row
    int K;           // words per plane row (multiple of 4)
    int Kg;          // 128-site groups per row (K / 4)
    int passes;      // colour classes per sweep
    int64_t row_words;   // P * K
    int64_t total_words; // (H + 2) * row_words
};

struct DevRng {
    uint32_t k0, k1;      // Philox key = seed
    uint32_t stream;
};

struct ThrView {
    int kind;               // ThrKind
    uint32_t scalar;        // THR_SCALAR
    int kmax;               // last plane that can decide a scalar compare
    const uint32_t* planes; // THR_SITE: [H][npar][32][K] threshold bit planes
    uint32_t tmask[32];     // THR_TABLE: bit idx of tmask[k] = bit 31-k of t16[idx]
    int cpol;               // THR_TABLE: -1, or a 4-bit polarity p with t16[idx] = t5[popc(idx ^ p)]
    uint32_t t5[5];
};

// Height propagation plan (per height-grid row): domain interval
// [xlo, xhi] (empty if xlo > xhi) and the spine column linking the row to
// the previous non-empty one (-1 for the first).
struct HeightPlan {
    int hw, hh;
};

// ---- kernel launchers (tl_kernels.cu); all return cudaError_t as int ----
int launch_pack(const Geom& g, const uint8_t* canon_dev, uint32_t* rows, void* stream);
int launch_unpack(const Geom& g, const uint32_t* rows, uint8_t* canon_dev, void* stream);
// `pass`: the colour class updated; `slot`: the pass slot that keys the
// random numbers (equal unless the pass order is random).
// flips: accepted-flip counter (nullptr = not counted).
int launch_pass_global(const Geom& g, uint32_t* rows, uint32_t pass, uint32_t slot, uint32_t sweep,
                       const DevRng& rng, const ThrView& th, const int2* grange, unsigned long long* flips,
                       void* stream);
int launch_hash(const Geom& g, const uint32_t* rows, unsigned long long* out, void* stream);
// Density counters are bit-sliced planes [32][H][row_words] (cplanes);
// launch_density_decode writes the canonical counts [ntype][H][W] from them.
int launch_density_accumulate(const Geom& g, const uint32_t* rows, uint32_t* cplanes, void* stream);
int launch_density_decode(const Geom& g, const uint32_t* cplanes, uint64_t samples, uint32_t* counts, void* stream);
int launch_density_read(const uint32_t* counts, uint64_t n, uint64_t samples, double* out,
                        void* stream);
int launch_nsew(const Geom& g, const uint32_t* counts, uint64_t samples, int kappa, double* out,
                void* stream);
// Domino shuffling of the Aztec diamond of order n: A, B, F are zeroed
// device scratch of 2n rows of (2n rounded up to 4) bytes each, rng a device
// copy of the key, canon the zeroed [2][2n+1][2n+1] output; status is raised
// if a created block is not a 2x2 hole.  Capturable into a graph.
int launch_shuffle(int n, uint8_t* A, uint8_t* B, uint8_t* F, const DevRng* rng, int* status, uint8_t* canon,
                   void* stream);
// seg: [nseg][6] height segments (y, lo, hi, parent, xs, dir); base_scratch: nseg ints.
int launch_height(const Geom& g, const uint32_t* rows, const int* seg, int nseg, int hw, int hh,
                  int32_t* out, int* base_scratch, void* stream);
int launch_threshold_planes(const Geom& g, const uint32_t* t_site_dev, uint32_t* planes,
                            void* stream);
// Device-generated log-normal weights -> per-site thresholds [H][W].
int launch_lognormal_thresholds(int lattice, int W, int H, double sigma, uint64_t seed, uint32_t* t, void* stream);
// Height with its segment-offset scratch in a static device array (no
// allocation); noalloc_prepare looks up the array's device address once per
// device (called when a context is created).
int noalloc_height_max_segments();
int noalloc_prepare(int device);
int launch_height_noalloc(const Geom& g, const uint32_t* rows, const int* seg, int nseg, int hw, int hh,
                          int32_t* out, int device, void* stream);

// Resident multi-sweep kernel.  One cooperative launch runs `nsweeps`
// sweeps from absolute sweep `sweep0`.  CTA c owns the rows
// [stripe_lo[c], stripe_lo[c+1]) and keeps them, plus `halo` rows on each
// side, in shared memory for the whole launch.  Every `halo` passes the
// CTAs publish their boundary rows and read their neighbours' (double
// buffered, ordered by per-CTA progress flags); in between, the halo rows
// are recomputed redundantly, the valid region shrinking by one row per pass.
struct ResidentPlan {
    int ctas;                      // cooperative grid size
    int threads;                   // threads per CTA (512 or 1024)
    int halo;                      // passes per exchange cycle (= halo rows per side)
    int npre;                      // random planes generated ahead per group
    int cap_items;                 // item-table capacity per CTA
    int cap_cycle;                 // groups touched per cycle, per CTA (upper bound)
    bool fast;                     // dominoes at t = 2^31: branch-free single-plane update
    size_t smem_bytes;             // dynamic shared memory per CTA
    const int* stripe_lo;          // device [ctas + 1]
    unsigned long long* xbuf;      // device [ctas][2][2][halo][row_words] tagged words
    int* status;                   // device error word: 0 ok, 1 a bounded wait gave up
};

// Shared-memory attribute and occupancy for the resident kernel of this
// lattice / threshold kind: blocks that fit on one SM (0 if none).
int resident_prepare(const Geom& g, int thr_kind, int threads, bool fast, size_t smem_bytes, int* blocks_per_sm);

// ring: per-sweep hashes (nullptr = off; must be zeroed).  counts: density
// counters sampled after every sweep s with s + 1 >= burn and
// (s + 1 - burn) % stride == 0 (nullptr or stride 0 = off).
int launch_resident(const Geom& g, uint32_t* rows, const ResidentPlan& plan, uint32_t sweep0,
                    uint32_t nsweeps, const DevRng& rng, const ThrView& th, const int2* grange,
                    unsigned int epoch, unsigned long long* ring, uint32_t* counts, uint64_t burn,
                    uint32_t stride, const uint8_t* colours, unsigned long long* flips, void* stream);
// Colours of the pass slots of nsweeps sweeps under the random pass order.
int launch_slot_colours(uint8_t* out, uint32_t sweep0, uint32_t nsweeps, int passes, const DevRng& rng, void* stream);

// Register-resident domino kernel at t = 2^31 (tl_regdom.cu).  Stripes of
// whole row pairs (2q, 2q + 1); pair q holds groups [hull[q].x, hull[q].y)
// (every group where its rows have sites or edges of domain faces, or the
// row above has sites); one thread per held group of the stripe and of
// `halo` rows on each side.
struct RegPlan {
    int ctas;
    int threads;                   // threads per CTA (<= 512, multiple of 32)
    int halo;                      // even
    size_t smem_bytes;
    const int* stripe_lo;          // device [ctas + 1], even
    const int2* hull;              // device [pairs]
    unsigned long long* xbuf;      // device [ctas][2][2][halo / 2][16][Kg][2]
    int* status;
};
size_t regdom_smem_bytes(int threads, int max_local_pairs);
int regdom_prepare(int threads, size_t smem_bytes, int* blocks_per_sm);
int launch_regdom(const Geom& g, uint32_t* rows, const RegPlan& plan, uint32_t sweep0, uint32_t nsweeps,
                  const DevRng& rng, unsigned int epoch, unsigned long long* ring, uint32_t* counts, uint64_t burn,
                  uint32_t stride, const uint8_t* colours, unsigned long long* flips, void* stream);

// ---- batched chains (tl_batch.cu) ----
struct BatchChain {
    Geom g;
    uint32_t* rows[2];          // two packed state buffers (ping-pong), each with pad rows
    const int2* grange;
    ThrView th;
    DevRng rng;
    uint32_t* sweep_base;       // device counter: absolute sweep of the next launch block
};
struct BatchTile {
    int chain, lo, hi;          // owned rows [lo, hi) of chain `chain`
};
// threads per tile: 256 or 128
int batch_prepare(size_t smem_bytes, int threads, int* blocks_per_sm);
// status: device int raised if a bounded wait for a tile's bulk copy gave up.
int launch_batch(const BatchChain* chains, const BatchTile* tiles, int ntiles, int R, uint32_t sweep_off, int src,
                 unsigned int* cursor, int grid, int threads, size_t smem_bytes, int* status, void* stream);
// advance every chain's sweep counter by k and zero the launch cursors
int launch_batch_advance(const BatchChain* chains, int nchains, uint32_t k, unsigned int* cursors, int ncursors,
                         void* stream);
int launch_batch_hash(const BatchChain* chains, const BatchTile* tiles, int ntiles, int buf,
                      unsigned long long* out, void* stream);
int launch_batch_copy(const BatchChain* chains, const BatchTile* tiles, int ntiles, int from, void* stream);

// Validation of a canonical state on the device (tl_kernels.cu): *first is
// ~0 if valid, else (kind << 48 | position) of the first failure; `aux` is
// the domain's cover (dominoes, lozenges) or boundary edges (six-vertex).
int launch_validate(const Geom& g, const uint8_t* canon, const uint8_t* aux, unsigned long long* first, void* stream);

// Debug words of the kernel files (debug build, -DTL_DEBUG): failures, then
// the id, index and bound of the first failed bounds check; each returns
// cudaErrorNotSupported in the normal build.  dbg_selftest runs one check
// on an out-of-range index (id 999) without the access it guards.
int dbg_fetch_kernels(unsigned long long* out, bool clear);
int dbg_fetch_regdom(unsigned long long* out, bool clear);
int dbg_fetch_resident(unsigned long long* out, bool clear);
int dbg_fetch_batch(unsigned long long* out, bool clear);
int dbg_fetch_shuffle(unsigned long long* out, bool clear);
int dbg_selftest();

}  // namespace tl
