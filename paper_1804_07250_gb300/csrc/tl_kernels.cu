// CUDA kernels for colour-class-parallel heat-bath Glauber dynamics on
// bit-packed tilings (Keating & Sridhar, "Random Tilings with the GPU",
// Sec. 1.1.3 cluster rotations, Sec. 1.2.1 lozenges, Sec. 1.2.4 six-vertex,
// Sec. 2.2 Rotate / Update kernels).  Written for sm_103a.
//
// Every thread updates one 128-site group (four 32-bit words, one Philox
// output) of one colour class in one row: the flippable mask is built with
// bitwise logic over the four neighbouring edge words, the heat-bath draw
// compares a bit-plane transposed Philox stream against the threshold MSB
// first and stops as soon as every flippable site is decided, and the flip is
// applied as an XOR of the four (or six) edge words.  Because each edge has a
// single owner inside a pass, there are no write conflicts except for the one
// word that straddles two groups when a plane is shifted by one site; that
// word is updated with atomicXor.  The paper's second kernel (UpdateBlack /
// UpdateWhite, which rebuilt the redundant 4-bit states of the other colour)
// has no counterpart: the packed state stores every edge once.
#include "tl_device.cuh"

#include <cstdint>
#include <mutex>

namespace tl {

// ---------------------------------------------------------------------------
// One launch per pass, state in global memory (L2-resident for mid sizes).
// Thread = (site row, group).  grange[y] = [first, last+1) groups of row y
// that hold sites of the domain.
// ---------------------------------------------------------------------------
template <int LAT, int TK>
__global__ void __launch_bounds__(256) pass_global_kernel(uint32_t* __restrict__ rows0, Geom g,
                                                          uint32_t pass, uint32_t slot, uint32_t sweep,
                                                          DevRng rng, ThrView th,
                                                          const int2* __restrict__ grange,
                                                          unsigned long long* __restrict__ flips)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int nrow = (LAT == LAT_SIXV) ? ((g.H + 1) >> 1) : g.H;
    const int rix = tid / g.Kg;
    const int m = tid - rix * g.Kg;
    if (rix >= nrow) return;
    int y, rr;
    if (LAT == LAT_SIXV) {
        y = 2 * rix + sixv_py(pass);
        if (y < 1 || y > g.N - 1) return;
        rr = rix;
    } else {
        y = rix;
        rr = y;
    }
#ifdef TL_DEBUG
    if (!TL_IN(y, g.H, 401)) return;
#endif
    const int2 gr = grange[y];
    if (m < gr.x || m >= gr.y) return;
#ifdef TL_DEBUG
    if (!TL_IN(4 * m + 3, g.K, 402)) return;
#endif
    const uint32_t grp = (uint32_t)(rr * g.Kg + m);
    uint32_t* row = rows0 + (int64_t)y * g.row_words;
    const RndPhilox rnd{grp, sweep, slot, rng};
    uint32_t nfl = 0;
    group_update<LAT, TK>(row, g.row_words, g, y, m, pass, rnd, th, nullptr, nullptr, flips ? &nfl : nullptr);
    if (nfl) atomicAdd(flips, (unsigned long long)nfl);
}

static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

int launch_pass_global(const Geom& g, uint32_t* rows, uint32_t pass, uint32_t slot, uint32_t sweep,
                       const DevRng& rng, const ThrView& th, const int2* grange, unsigned long long* flips,
                       void* stream)
{
    const int nrow = (g.lattice == LAT_SIXV) ? ((g.H + 1) >> 1) : g.H;
    const int64_t threads = (int64_t)nrow * g.Kg;
    const int blocks = (int)((threads + 255) / 256);
    uint32_t* rows0 = rows + g.row_words;
    if (g.lattice == LAT_DOMINO) {
        if (th.kind == THR_SITE)
            pass_global_kernel<LAT_DOMINO, THR_SITE><<<blocks, 256, 0, S(stream)>>>(rows0, g, pass, slot, sweep, rng, th, grange, flips);
        else
            pass_global_kernel<LAT_DOMINO, THR_SCALAR><<<blocks, 256, 0, S(stream)>>>(rows0, g, pass, slot, sweep, rng, th, grange, flips);
    } else if (g.lattice == LAT_LOZENGE) {
        if (th.kind == THR_SITE)
            pass_global_kernel<LAT_LOZENGE, THR_SITE><<<blocks, 256, 0, S(stream)>>>(rows0, g, pass, slot, sweep, rng, th, grange, flips);
        else
            pass_global_kernel<LAT_LOZENGE, THR_SCALAR><<<blocks, 256, 0, S(stream)>>>(rows0, g, pass, slot, sweep, rng, th, grange, flips);
    } else {
        pass_global_kernel<LAT_SIXV, THR_TABLE><<<blocks, 256, 0, S(stream)>>>(rows0, g, pass, slot, sweep, rng, th, grange, flips);
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout conversion.  Canonical: uint8 [ntype][H][W].
// ---------------------------------------------------------------------------
__global__ void pack_kernel(const uint8_t* __restrict__ canon, uint32_t* __restrict__ rows, Geom g)
{
    const int64_t n = (int64_t)g.H * g.row_words;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / g.row_words);
        const int rem = (int)(i - (int64_t)y * g.row_words);
        const int pl = rem / g.K, k = rem - pl * g.K;
        const int type = pl / g.npar, res = pl - type * g.npar;
        const uint8_t* src = canon + ((size_t)type * g.H + y) * g.W;
        uint32_t w = 0;
        for (int b = 0; b < 32; ++b) {
            const int x = g.npar * (32 * k + b) + res;
            if (x < g.W && src[x]) w |= 1u << b;
        }
        rows[g.row_words + i] = w;
    }
}

__global__ void unpack_kernel(const uint32_t* __restrict__ rows, uint8_t* __restrict__ canon, Geom g)
{
    const int64_t n = (int64_t)g.ntype * g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.W);
        const int64_t r = i / g.W;
        const int y = (int)(r % g.H);
        const int type = (int)(r / g.H);
        const int res = x % g.npar, j = x / g.npar;
        const uint32_t w = rows[g.row_words + (int64_t)y * g.row_words +
                                (int64_t)(type * g.npar + res) * g.K + (j >> 5)];
        canon[i] = (uint8_t)((w >> (j & 31)) & 1u);
    }
}

static int grid_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 152 * 32) b = 152 * 32;
    if (b < 1) b = 1;
    return (int)b;
}

int launch_pack(const Geom& g, const uint8_t* canon_dev, uint32_t* rows, void* stream)
{
    cudaError_t e = cudaMemsetAsync(rows, 0, (size_t)g.total_words * 4, S(stream));
    if (e != cudaSuccess) return (int)e;
    const int64_t n = (int64_t)g.H * g.row_words;
    pack_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(canon_dev, rows, g);
    return (int)cudaGetLastError();
}

int launch_unpack(const Geom& g, const uint32_t* rows, uint8_t* canon_dev, void* stream)
{
    const int64_t n = (int64_t)g.ntype * g.H * g.W;
    unpack_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(rows, canon_dev, g);
    return (int)cudaGetLastError();
}

// Per-site thresholds [H][W] -> bit planes [H][npar][32][K]; plane k holds
// bit (31-k) of t for each site of the (row, residue) plane row.
__global__ void threshold_planes_kernel(const uint32_t* __restrict__ t, uint32_t* __restrict__ planes, Geom g)
{
    const int64_t n = (int64_t)g.H * g.npar * g.K;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i % g.K);
        const int64_t r = i / g.K;
        const int res = (int)(r % g.npar);
        const int y = (int)(r / g.npar);
        uint32_t tv[32];
        for (int b = 0; b < 32; ++b) {
            const int x = g.npar * (32 * k + b) + res;
            tv[b] = (x < g.W) ? t[(size_t)y * g.W + x] : 0u;
        }
        uint32_t* out = planes + ((size_t)(y * g.npar + res) * 32) * g.K + k;
        for (int pl = 0; pl < 32; ++pl) {
            uint32_t w = 0;
            for (int b = 0; b < 32; ++b) w |= ((tv[b] >> (31 - pl)) & 1u) << b;
            out[(size_t)pl * g.K] = w;
        }
    }
}

int launch_threshold_planes(const Geom& g, const uint32_t* t_site_dev, uint32_t* planes, void* stream)
{
    const int64_t n = (int64_t)g.H * g.npar * g.K;
    threshold_planes_kernel<<<grid_for(n, 128), 128, 0, S(stream)>>>(t_site_dev, planes, g);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Validation of a canonical state against its domain, on the device: every
// byte 0 or 1; dominoes: no edge outside the box, every face of the domain
// covered once and no other; lozenges: every triangle covered as the domain
// says; six-vertex: no bit off the lattice, the external edges those of the
// boundary, the ice rule at every vertex.  The first failure in the order of
// a row-major scan (kinds in this order) is kept as the smallest code
// (kind << 48 | position) by an atomic min; *first stays ~0 if the state is
// valid.  Kinds: 1 byte (position = byte index), 2 domino edge right of the
// box (y), 3 domino edge above the box (x), 4 domino face (y (W-1) + x),
// 5 lozenge triangles ((y+1)(W+1) + x+1), 6 six-vertex bit off the lattice
// (Y W + X), 7 six-vertex boundary (k), 8 six-vertex ice rule (Y W + X).
// ---------------------------------------------------------------------------
struct DevCanon {
    const uint8_t* s;
    int W, H;
    TL_DEV int at(int type, int x, int y) const
    {
        if (x < 0 || y < 0 || x >= W || y >= H) return 0;
        return s[((size_t)type * H + y) * W + x];
    }
};

TL_DEV void vfail(unsigned long long* first, int kind, uint64_t pos)
{
    atomicMin(first, ((unsigned long long)kind << 48) | (unsigned long long)pos);
}

__global__ void validate_bytes_kernel(const uint8_t* __restrict__ s, size_t n, unsigned long long* first)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        if (s[i] > 1) vfail(first, 1, i);
}

// aux: face cover [(H-1)][(W-1)]
__global__ void validate_domino_kernel(const uint8_t* __restrict__ s, Geom g, const uint8_t* __restrict__ cover,
                                       unsigned long long* first)
{
    const DevCanon c{s, g.W, g.H};
    const int64_t nf = (int64_t)(g.W - 1) * (g.H - 1);
    const int64_t nall = nf + g.H + g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nall; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < g.H) {
            if (c.at(0, g.W - 1, (int)i)) vfail(first, 2, (uint64_t)i);
        } else if (i < g.H + g.W) {
            if (c.at(1, (int)(i - g.H), g.H - 1)) vfail(first, 3, (uint64_t)(i - g.H));
        } else {
            const int64_t f = i - g.H - g.W;
            const int y = (int)(f / (g.W - 1)), x = (int)(f - (int64_t)y * (g.W - 1));
            const int k = c.at(0, x, y) + c.at(0, x, y + 1) + c.at(1, x, y) + c.at(1, x + 1, y);
            if (k != cover[f]) vfail(first, 4, (uint64_t)f);
        }
    }
}

// aux: triangle cover, up then down, [(H+1)][(W+1)] each
__global__ void validate_lozenge_kernel(const uint8_t* __restrict__ s, Geom g, const uint8_t* __restrict__ cover,
                                        unsigned long long* first)
{
    const DevCanon c{s, g.W, g.H};
    const int TW = g.W + 1, TH = g.H + 1;
    const int64_t nt = (int64_t)TW * TH;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / TW) - 1, x = (int)(i % TW) - 1;
        const int u = c.at(0, x, y) + c.at(1, x + 1, y) + c.at(2, x, y);
        const int v = c.at(2, x, y) + c.at(1, x, y) + c.at(0, x, y + 1);
        if (u != cover[i] || v != cover[nt + i]) vfail(first, 5, (uint64_t)i);
    }
}

// aux: the boundary edges of the domain, [4][N]: for k = 1..N (index k - 1)
// type 0 at (0, k), type 0 at (N, k), type 1 at (k, 0), type 1 at (k, N)
__global__ void validate_sixv_kernel(const uint8_t* __restrict__ s, Geom g, const uint8_t* __restrict__ bnd,
                                     unsigned long long* first)
{
    const DevCanon c{s, g.W, g.H};
    const int N = g.N;
    const int64_t nb = (int64_t)g.W * g.H;
    const int64_t nall = nb + N + nb;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nall; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < nb) {
            const int Y = (int)(i / g.W), X = (int)(i % g.W);
            const bool hreal = Y >= 1 && Y <= N && X <= N;
            const bool vreal = X >= 1 && X <= N && Y <= N;
            if ((c.at(0, X, Y) && !hreal) || (c.at(1, X, Y) && !vreal)) vfail(first, 6, (uint64_t)i);
        } else if (i < nb + N) {
            const int k = (int)(i - nb) + 1;
            if (c.at(0, 0, k) != bnd[k - 1] || c.at(0, N, k) != bnd[N + k - 1] || c.at(1, k, 0) != bnd[2 * N + k - 1] ||
                c.at(1, k, N) != bnd[3 * N + k - 1])
                vfail(first, 7, (uint64_t)k);
        } else {
            const int64_t j = i - nb - N;
            const int Y = (int)(j / g.W), X = (int)(j % g.W);
            if (Y < 1 || Y > N || X < 1 || X > N) continue;
            const int L = c.at(0, X - 1, Y), R = c.at(0, X, Y), D = c.at(1, X, Y - 1), U = c.at(1, X, Y);
            if (L + U != D + R) vfail(first, 8, (uint64_t)j);
        }
    }
}

int launch_validate(const Geom& g, const uint8_t* canon, const uint8_t* aux, unsigned long long* first, void* stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(first, 0xFF, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return (int)e;
    const size_t n = (size_t)g.ntype * g.W * g.H;
    validate_bytes_kernel<<<grid_for((int64_t)n, 256), 256, 0, st>>>(canon, n, first);
    if (g.lattice == LAT_DOMINO)
        validate_domino_kernel<<<grid_for((int64_t)(g.W - 1) * (g.H - 1) + g.W + g.H, 256), 256, 0, st>>>(canon, g, aux, first);
    else if (g.lattice == LAT_LOZENGE)
        validate_lozenge_kernel<<<grid_for((int64_t)(g.W + 1) * (g.H + 1), 256), 256, 0, st>>>(canon, g, aux, first);
    else
        validate_sixv_kernel<<<grid_for((int64_t)2 * g.W * g.H + g.N, 256), 256, 0, st>>>(canon, g, aux, first);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Observables.
// ---------------------------------------------------------------------------
__global__ void hash_kernel(const uint32_t* __restrict__ rows0, Geom g, unsigned long long* out)
{
    const int64_t n = (int64_t)g.H * g.row_words;
    uint64_t acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = rows0[i];
        if (!w) continue;
        const int y = (int)(i / g.row_words);
        const int rem = (int)(i - (int64_t)y * g.row_words);
        const int pl = rem / g.K, k = rem - pl * g.K;
        acc += word_hash(w, g, y, pl, k);
    }
    for (int off = 16; off; off >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, off);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, (unsigned long long)acc);
}

int launch_hash(const Geom& g, const uint32_t* rows, unsigned long long* out, void* stream)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), S(stream));
    if (e != cudaSuccess) return (int)e;
    const int64_t n = (int64_t)g.H * g.row_words;
    hash_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(rows + g.row_words, g, out);
    return (int)cudaGetLastError();
}

// Edge-occupancy counters, bit-sliced in the packed layout (word_count_sliced).
__global__ void density_acc_kernel(const uint32_t* __restrict__ rows0, Geom g, uint32_t* __restrict__ cplanes)
{
    const int64_t n = (int64_t)g.H * g.row_words;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t w = rows0[i];
        if (w) word_count_sliced(w, i, n, cplanes);
    }
}

int launch_density_accumulate(const Geom& g, const uint32_t* rows, uint32_t* cplanes, void* stream)
{
    const int64_t n = (int64_t)g.H * g.row_words;
    density_acc_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(rows + g.row_words, g, cplanes);
    return (int)cudaGetLastError();
}

// Canonical counters counts[type][y][x] from the bit-sliced planes; only the
// `nbits` low planes can be non-zero (samples < 2^nbits).
__global__ void density_decode_kernel(const uint32_t* __restrict__ cplanes, Geom g, int nbits,
                                      uint32_t* __restrict__ counts)
{
    const int64_t n = (int64_t)g.ntype * g.H * g.W, plane = (int64_t)g.H * g.row_words;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.W);
        const int64_t r = i / g.W;
        const int y = (int)(r % g.H), type = (int)(r / g.H);
        const int res = x % g.npar, j = x / g.npar;
        const int64_t w = (int64_t)y * g.row_words + (int64_t)(type * g.npar + res) * g.K + (j >> 5);
        uint32_t v = 0;
        for (int b = 0; b < nbits; ++b) v |= ((cplanes[(int64_t)b * plane + w] >> (j & 31)) & 1u) << b;
        counts[i] = v;
    }
}

int launch_density_decode(const Geom& g, const uint32_t* cplanes, uint64_t samples, uint32_t* counts, void* stream)
{
    int nbits = 0;
    while (nbits < 32 && (samples >> nbits)) ++nbits;
    const int64_t n = (int64_t)g.ntype * g.H * g.W;
    density_decode_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(cplanes, g, nbits, counts);
    return (int)cudaGetLastError();
}

__global__ void density_read_kernel(const uint32_t* __restrict__ counts, uint64_t n, double inv,
                                    double* __restrict__ out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = (double)counts[i] * inv;
}

int launch_density_read(const uint32_t* counts, uint64_t n, uint64_t samples, double* out, void* stream)
{
    const double inv = samples ? 1.0 / (double)samples : 0.0;
    density_read_kernel<<<grid_for((int64_t)n, 256), 256, 0, S(stream)>>>(counts, n, inv, out);
    return (int)cudaGetLastError();
}

// Domino type densities per face from the edge counters.  Face (x,y) of
// colour c = (x+y) mod 2 is covered by a domino crossing exactly one of its
// edges: right Vt(x+1,y) or left Vt(x,y) (horizontal), top Hz(x,y+1) or
// bottom Hz(x,y) (vertical).  Horizontal: north iff the left square has
// colour kappa.  Vertical: west iff the bottom square has colour != kappa.
__global__ void nsew_kernel(const uint32_t* __restrict__ counts, Geom g, double inv, int kappa,
                            double* __restrict__ out)
{
    const int FW = g.W - 1, FH = g.H - 1;
    const int64_t n = (int64_t)FW * FH;
    const uint32_t* hz = counts;
    const uint32_t* vt = counts + (size_t)g.H * g.W;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(i % FW), y = (int)(i / FW);
        const int c = (x + y) & 1;
        const double right = vt[(size_t)y * g.W + x + 1], left = vt[(size_t)y * g.W + x];
        const double top = hz[(size_t)(y + 1) * g.W + x], bottom = hz[(size_t)y * g.W + x];
        double nn = 0, ss = 0, ee = 0, ww = 0;
        if (c == kappa) nn += right; else ss += right;          // this face is the left square
        if ((1 - c) == kappa) nn += left; else ss += left;      // left square is the neighbour
        if (c != kappa) ww += top; else ee += top;              // this face is the bottom square
        if ((1 - c) != kappa) ww += bottom; else ee += bottom;  // bottom square is the neighbour
        out[i] = nn * inv;
        out[n + i] = ss * inv;
        out[2 * n + i] = ee * inv;
        out[3 * n + i] = ww * inv;
    }
}

int launch_nsew(const Geom& g, const uint32_t* counts, uint64_t samples, int kappa, double* out, void* stream)
{
    const double inv = samples ? 1.0 / (double)samples : 0.0;
    const int64_t n = (int64_t)(g.W - 1) * (g.H - 1);
    nsew_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(counts, g, inv, kappa, out);
    return (int)cudaGetLastError();
}

// Height function: (1) prefix sums of horizontal steps along each segment
// of a row, (2) one block links every segment to its parent through a
// vertical step and accumulates the offsets, (3) offsets are added.
TL_DEV uint32_t bit_at(const uint32_t* rows0, const Geom& g, int type, int x, int y)
{
    if (x < 0 || y < 0 || x >= g.W || y >= g.H) return 0u;
    const int res = x % g.npar, j = x / g.npar;
    const uint32_t w = rows0[(int64_t)y * g.row_words + (int64_t)(type * g.npar + res) * g.K + (j >> 5)];
    return (w >> (j & 31)) & 1u;
}

// Step from grid point (x,y) to (x+1,y) / from (x,y-1) to (x,y).
TL_DEV int hstep(const uint32_t* rows0, const Geom& g, int x, int y)
{
    if (g.lattice == LAT_DOMINO) {
        const int s = ((x + y) & 1) ? -1 : 1;
        return bit_at(rows0, g, 0, x, y) ? -3 * s : s;
    }
    if (g.lattice == LAT_LOZENGE) return -(int)bit_at(rows0, g, 0, x, y);
    return bit_at(rows0, g, 1, x + 1, y) ? 1 : -1;   // faces: cross Vt(x+1, y)
}
TL_DEV int vstep(const uint32_t* rows0, const Geom& g, int x, int y)
{
    if (g.lattice == LAT_DOMINO) {
        const int s = ((x - 1 + y - 1) & 1) ? -1 : 1;
        return bit_at(rows0, g, 1, x, y - 1) ? -3 * s : s;
    }
    if (g.lattice == LAT_LOZENGE) return -(int)bit_at(rows0, g, 1, x, y - 1);
    return bit_at(rows0, g, 0, x, y) ? 1 : -1;       // faces: cross Hz(x, y)
}

// Height segments: seg[6 s .. 6 s + 5] = (y, lo, hi, parent, xs, dir): a
// maximal run [lo, hi] of row y joined by domain steps, the segment it is
// linked to (-1 for the first, which holds the reference vertex) and the
// column xs of the linking vertical step, dir = +1 if this segment lies one
// row above its parent and -1 if below.  Parents precede children.
__global__ void height_fill_kernel(int32_t* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = INT32_MIN;
}

// Heights along each segment relative to its left end.
__global__ void __launch_bounds__(256) height_seg_kernel(const uint32_t* __restrict__ rows0, Geom g,
                                                         const int* __restrict__ seg, int hw,
                                                         int32_t* __restrict__ out)
{
    const int* sg = seg + 6 * (size_t)blockIdx.x;
    const int y = sg[0], lo = sg[1], hi = sg[2];
#ifdef TL_DEBUG
    // a segment of row y spans vertices lo .. hi of a row of hw heights
    if (!(TL_IN(y, g.H, 403) && TL_IN(lo, hw, 404) && TL_IN(hi, hw, 404))) return;
#endif
    int32_t* o = out + (size_t)y * hw;
    __shared__ int part[256];
    const int n = hi - lo + 1;
    const int per = (n + 255) / 256;
    const int a = lo + threadIdx.x * per;
    int sum = 0;
    for (int i = 0; i < per; ++i) {
        const int x = a + i;
        if (x < hi) sum += hstep(rows0, g, x, y);   // step x -> x+1
    }
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
        const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;   // height of x = a relative to lo
    for (int i = 0; i < per; ++i) {
        const int x = a + i;
        if (x <= hi) {
            o[x] = run;
            if (x < hi) run += hstep(rows0, g, x, y);
        }
    }
}

// Offsets of the segments: the differences to the parents in parallel, then
// one thread accumulates them in parent-first order.
__global__ void __launch_bounds__(1024) height_link_kernel(const uint32_t* __restrict__ rows0, Geom g,
                                                           const int* __restrict__ seg, int nseg, int hw,
                                                           const int32_t* __restrict__ rel, int* __restrict__ base)
{
    __shared__ int dd[1024], par[1024];
    int last = 0;
    for (int c0 = 0; c0 < nseg; c0 += 1024) {
        const int s = c0 + threadIdx.x;
        if (s < nseg) {
            const int* sg = seg + 6 * (size_t)s;
            const int y = sg[0], p = sg[3], xs = sg[4], dir = sg[5];
            int d = 0;
            if (p >= 0) {
                const int py = seg[6 * (size_t)p];
                const int step = dir > 0 ? vstep(rows0, g, xs, y) : -vstep(rows0, g, xs, y + 1);
                d = rel[(size_t)py * hw + xs] + step - rel[(size_t)y * hw + xs];
            }
            dd[threadIdx.x] = d;
            par[threadIdx.x] = p;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            const int n = nseg - c0 < 1024 ? nseg - c0 : 1024;
            for (int i = 0; i < n; ++i) {
                const int s2 = c0 + i, p = par[i];
                const int b = p < 0 ? 0 : (p == s2 - 1 ? last : base[p]);
                last = b + dd[i];
                base[s2] = last;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) height_add_kernel(int32_t* __restrict__ out, const int* __restrict__ seg,
                                                         const int* __restrict__ base, int hw)
{
    const int* sg = seg + 6 * (size_t)blockIdx.x;
    const int y = sg[0], lo = sg[1], hi = sg[2];
    const int b = base[blockIdx.x];
    int32_t* o = out + (size_t)y * hw;
    for (int x = lo + threadIdx.x; x <= hi; x += 256) o[x] += b;
}

int launch_height(const Geom& g, const uint32_t* rows, const int* seg, int nseg, int hw, int hh, int32_t* out,
                  int* base_scratch, void* stream)
{
    const uint32_t* rows0 = rows + g.row_words;
    height_fill_kernel<<<grid_for((int64_t)hw * hh, 256), 256, 0, S(stream)>>>(out, (int64_t)hw * hh);
    if (nseg > 0) {
        height_seg_kernel<<<nseg, 256, 0, S(stream)>>>(rows0, g, seg, hw, out);
        height_link_kernel<<<1, 1024, 0, S(stream)>>>(rows0, g, seg, nseg, hw, out, base_scratch);
        height_add_kernel<<<nseg, 256, 0, S(stream)>>>(out, seg, base_scratch, hw);
    }
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Generated log-normal weights and their heat-bath thresholds, on the device.
// Weight of item i (an edge or a vertex, by canonical index) = exp(sigma Z),
// Z standard normal by the Box-Muller transform of two 32-bit words of
// Philox4x32-10(key = seed, counter = (i lo, i hi, 0x6C6F676E, 0)).  The
// threshold arithmetic uses correctly rounded FP64 operations in the order of
// the host formulas (no fused multiply-add), so for equal weights it equals
// the host result bit for bit.
// ---------------------------------------------------------------------------
TL_DEV double lognormal_weight(uint64_t i, double sigma, uint32_t k0, uint32_t k1)
{
    const uint4 o = philox10((uint32_t)i, (uint32_t)(i >> 32), 0x6C6F676Eu, 0u, k0, k1);
    const double u1 = ((double)o.x + 1.0) * (1.0 / 4294967296.0);   // (0, 1]
    const double u2 = (double)o.y * (1.0 / 4294967296.0);           // [0, 1)
    const double z = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    return exp(sigma * z);
}

TL_DEV uint32_t prob_threshold(double p)
{
    const double t = floor(__dmul_rn(p, 4294967296.0));
    if (!(t > 0.0)) return 0u;
    if (t >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)t;
}

// Dominoes: edge weights on the canonical [2][H][W] layout; t at every vertex
// from up = wE * wW, down = wN * wS, P = up / (up + down) (1.0 off the box).
__global__ void lognormal_domino_kernel(int W, int H, double sigma, uint32_t k0, uint32_t k1, uint32_t* t)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(v % W), y = (int)(v / W);
        auto wt = [&](int type, int xx, int yy) -> double {
            if (xx < 0 || yy < 0 || xx >= W || yy >= H) return 1.0;
            return lognormal_weight(((uint64_t)type * H + yy) * W + xx, sigma, k0, k1);
        };
        const double up = __dmul_rn(wt(0, x, y), wt(0, x - 1, y));
        const double down = __dmul_rn(wt(1, x, y), wt(1, x, y - 1));
        t[v] = prob_threshold(__ddiv_rn(up, __dadd_rn(up, down)));
    }
}

// Lozenges: volume weight q_v per vertex; P(add a cube) = q / (1 + q).
__global__ void lognormal_lozenge_kernel(int W, int H, double sigma, uint32_t k0, uint32_t k1, uint32_t* t)
{
    const int64_t n = (int64_t)W * H;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const double q = lognormal_weight((uint64_t)v, sigma, k0, k1);
        t[v] = prob_threshold(__ddiv_rn(q, __dadd_rn(1.0, q)));
    }
}

int launch_lognormal_thresholds(int lattice, int W, int H, double sigma, uint64_t seed, uint32_t* t, void* stream)
{
    const int64_t n = (int64_t)W * H;
    if (lattice == LAT_DOMINO)
        lognormal_domino_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(W, H, sigma, (uint32_t)seed,
                                                                       (uint32_t)(seed >> 32), t);
    else
        lognormal_lozenge_kernel<<<grid_for(n, 256), 256, 0, S(stream)>>>(W, H, sigma, (uint32_t)seed,
                                                                        (uint32_t)(seed >> 32), t);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Height function without any allocation.  For callers that cannot allocate
// device memory at the time they need the heights (for example code running
// under a memory budget that forbids cudaMalloc, or a real-time loop that
// must not synchronise the device the way cudaMalloc / cudaFree can), the
// per-segment offsets that launch_height keeps in chain-owned memory live here
// in one file-scope device array instead.  The array holds kNoAllocMaxSegs
// ints (256 KiB): one per height segment, a maximal run of domain vertices in
// one row (one segment per row for the Aztec diamond, rectangles, hexagons and
// the domain-wall square; a row of a non-convex domain from a boundary path
// can hold several).  Domains with more segments are rejected.  Every GPU
// that loads the library keeps the array until the process exits.  All calls
// on a device share it: each call rewrites every entry it reads, so nothing
// needs clearing, but calls whose kernels overlap on the GPU (concurrent
// streams) race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxSegs = 65536;
static __device__ __align__(256) int g_noalloc_height_base[kNoAllocMaxSegs];

constexpr int kNoAllocMaxDevices = 64;
static std::mutex g_noalloc_mu;
static int* g_noalloc_base_dev[kNoAllocMaxDevices];   // device address per device ordinal

int noalloc_height_max_segments() { return kNoAllocMaxSegs; }

// The device address of the scratch array must come from cudaGetSymbolAddress
// with the device current: in host code the symbol names a host-side stand-in.
// Looked up once per device, when a context is created on it (the lookup can
// load this module, which allocates), so the entry point itself never does.
int noalloc_prepare(int device)
{
    if (device < 0 || device >= kNoAllocMaxDevices) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_base_dev[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_height_base);
        if (e != cudaSuccess) return (int)e;
        g_noalloc_base_dev[device] = static_cast<int*>(p);
    }
    return 0;
}

static int noalloc_scratch(int device, int** out)
{
    if (device < 0 || device >= kNoAllocMaxDevices) return (int)cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    *out = g_noalloc_base_dev[device];
    return *out ? 0 : (int)cudaErrorInitializationError;
}

int launch_height_noalloc(const Geom& g, const uint32_t* rows, const int* seg, int nseg, int hw, int hh,
                          int32_t* out, int device, void* stream)
{
    if (nseg > kNoAllocMaxSegs) return (int)cudaErrorInvalidValue;
    int* base = nullptr;
    const int e = noalloc_scratch(device, &base);
    if (e) return e;
    return launch_height(g, rows, seg, nseg, hw, hh, out, base, stream);
}

// This file's debug word (failures, then the id, index and bound of the
// first failed check); cudaErrorNotSupported in the normal build.
int dbg_fetch_kernels(unsigned long long* out, bool clear)
{
#ifdef TL_DEBUG
    return tl_dbg_fetch(out, clear);
#else
    (void)out;
    (void)clear;
    return (int)cudaErrorNotSupported;
#endif
}

#ifdef TL_DEBUG
// One check on an index out of its range (5 of 3, id 999) and none of the
// access it guards: the failure must be recorded, nothing else happens.
__global__ void dbg_selftest_kernel(int* out)
{
    int x = 0;
    if (TL_IN(threadIdx.x + 5, 3, 999)) x = 1;
    out[threadIdx.x] = x;
}
#endif

int dbg_selftest()
{
#ifdef TL_DEBUG
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e == cudaSuccess) {
        dbg_selftest_kernel<<<1, 1>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d);
    return (int)e;
#else
    return (int)cudaErrorNotSupported;
#endif
}

}  // namespace tl
