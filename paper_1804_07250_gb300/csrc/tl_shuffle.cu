// Domino shuffling: exact uniform random tilings of the Aztec diamond (the
// shuffling algorithms the paper names as an alternative exact sampler,
// Sec. 3; Elkies, Kuperberg, Larsen and Propp).
//
// Cells are unit squares with lower-left corner (x, y), x, y in [-n, n); the
// diamond of order k holds the cells with |x + 1/2| + |y + 1/2| <= k.  A
// cell stores which part of a domino covers it (empty, left / right half of
// a horizontal domino, bottom / top half of a vertical one).  In order k a
// horizontal domino with left cell (x, y) goes north if x + y + k is even,
// else south; a vertical one with bottom cell (x, y) goes east if x + y + k
// is even, else west.  One step k -> k + 1 is three data-parallel kernels:
//  1. move (gather): every cell of order k + 1 looks at the four cells a
//     domino could arrive from, and takes the part of the one that moves in,
//     unless it is in a bad block (a north-going domino right below a
//     south-going one, or an east-going one right left of a west-going one);
//  2. mark: the cells left empty form disjoint 2x2 blocks whose lower-left
//     cells have x + y + k + 1 odd; an empty cell of that parity starts a
//     block iff the run of empty cells below it in its column has even
//     length;
//  3. create: each marked block gets two horizontal dominoes if its Philox
//     draw is below 2^31, else two vertical ones.
#include "tl_device.cuh"

#include <cstdint>

namespace tl {

enum : uint8_t { SH_EMPTY = 0, SH_HL = 1, SH_HR = 2, SH_VB = 3, SH_VT = 4 };

TL_DEV bool in_diamond(int x, int y, int k) { return abs(2 * x + 1) + abs(2 * y + 1) <= 2 * k; }

// Cell of this thread: block row blockIdx.y is diamond row y = blockIdx.y - K,
// whose cells are x in [-w, w) with w = K - |y + 1/2| + 1/2; threads past
// the row's end return false.
TL_DEV bool row_cell(int K, int& x, int& y)
{
    y = (int)blockIdx.y - K;
    const int w = K - (y >= 0 ? y : -y - 1);
    const int t = (int)(blockIdx.x * blockDim.x + threadIdx.x);
    x = t - w;
    return t < 2 * w;
}

TL_DEV uint8_t cell_at(const uint8_t* A, int n, int x, int y)
{
    if (x < -n || y < -n || x >= n || y >= n) return SH_EMPTY;
    return A[(size_t)(y + n) * (2 * n) + (x + n)];
}

// Whether the domino with anchor (left or bottom) cell (ax, ay) and
// orientation o (0 horizontal) of order k survives the destruction step.
TL_DEV bool survives(const uint8_t* A, int n, int k, int ax, int ay, int o)
{
    const bool even = ((ax + ay + k) & 1) == 0;
    if (o == 0) return even ? cell_at(A, n, ax, ay + 1) != SH_HL : cell_at(A, n, ax, ay - 1) != SH_HL;
    return even ? cell_at(A, n, ax + 1, ay) != SH_VB : cell_at(A, n, ax - 1, ay) != SH_VB;
}

__global__ void shuffle_move_kernel(const uint8_t* __restrict__ A, uint8_t* __restrict__ B, int n, int k)
{
    const int K = k + 1;
    int x, y;
    if (!row_cell(K, x, y)) return;
    {
        uint8_t out = SH_EMPTY;
        // from below, going north (horizontal)
        uint8_t c = cell_at(A, n, x, y - 1);
        if (c == SH_HL || c == SH_HR) {
            const int ax = c == SH_HL ? x : x - 1, ay = y - 1;
            if (((ax + ay + k) & 1) == 0 && survives(A, n, k, ax, ay, 0)) out = c;
        }
        c = cell_at(A, n, x, y + 1);   // from above, going south
        if (c == SH_HL || c == SH_HR) {
            const int ax = c == SH_HL ? x : x - 1, ay = y + 1;
            if (((ax + ay + k) & 1) == 1 && survives(A, n, k, ax, ay, 0)) out = c;
        }
        c = cell_at(A, n, x - 1, y);   // from the left, going east (vertical)
        if (c == SH_VB || c == SH_VT) {
            const int ax = x - 1, ay = c == SH_VB ? y : y - 1;
            if (((ax + ay + k) & 1) == 0 && survives(A, n, k, ax, ay, 1)) out = c;
        }
        c = cell_at(A, n, x + 1, y);   // from the right, going west
        if (c == SH_VB || c == SH_VT) {
            const int ax = x + 1, ay = c == SH_VB ? y : y - 1;
            if (((ax + ay + k) & 1) == 1 && survives(A, n, k, ax, ay, 1)) out = c;
        }
        B[(size_t)(y + n) * (2 * n) + (x + n)] = out;
    }
}

// Mark the lower-left cells of the holes' 2x2 blocks in F: an empty cell
// with x + y + K odd whose run of empty cells below it (in its column) has
// even length.  Blocks in a column are stacked from the bottom of each run,
// so this picks exactly one corner per block; runs are short, so each
// thread walks down its own run.
__global__ void shuffle_mark_kernel(const uint8_t* __restrict__ B, uint8_t* __restrict__ F, int n, int K)
{
    int x, y;
    if (!row_cell(K, x, y)) return;
    {
        const size_t c = (size_t)(y + n) * (2 * n) + (x + n);
        uint8_t mark = 0;
        if (B[c] == SH_EMPTY && ((x + y + K) & 1) == 1) {
            int below = 0;
            for (int yy = y - 1; yy >= -K && in_diamond(x, yy, K) &&
                                 B[(size_t)(yy + n) * (2 * n) + (x + n)] == SH_EMPTY;
                 --yy)
                ++below;
            mark = (below & 1) == 0;
        }
        F[c] = mark;
    }
}

__global__ void shuffle_create_kernel(uint8_t* __restrict__ B, const uint8_t* __restrict__ F, int n, int K,
                                      DevRng rng, uint32_t tbar, int* __restrict__ status)
{
    int x, y;
    if (!row_cell(K, x, y)) return;
    {
        const size_t c = (size_t)(y + n) * (2 * n) + (x + n);
        if (!F[c]) return;
        const size_t r = c + 1, u = c + 2 * n, ur = u + 1;
        if (x + 1 >= n || y + 1 >= n || B[r] != SH_EMPTY || B[u] != SH_EMPTY || B[ur] != SH_EMPTY) {
            atomicExch(status, 1);   // not a 2x2 hole: cannot happen for a valid tiling
            return;
        }
        const uint4 o = philox10(((uint32_t)(y + n) << 16) | (uint32_t)(x + n), (uint32_t)K, 0xFFFE0000u, rng.stream,
                                 rng.k0, rng.k1);
        if (o.x < tbar) {
            B[c] = SH_HL; B[r] = SH_HR; B[u] = SH_HL; B[ur] = SH_HR;
        } else {
            B[c] = SH_VB; B[u] = SH_VT; B[r] = SH_VB; B[ur] = SH_VT;
        }
    }
}

// Canonical domino state of the order-n diamond (box (2n+1)^2, zeroed):
// a horizontal domino crosses the vertical edge between its cells, a
// vertical one the horizontal edge.
__global__ void shuffle_canon_kernel(const uint8_t* __restrict__ A, int n, uint8_t* __restrict__ canon)
{
    const int S = 2 * n, W = 2 * n + 1;
    const int64_t total = (int64_t)S * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(i % S), cy = (int)(i / S);   // cell (cx - n, cy - n)
        const uint8_t v = A[i];
        if (v == SH_HL) canon[(size_t)W * W + (size_t)cy * W + cx + 1] = 1;    // Vt(x+1, y)
        else if (v == SH_VB) canon[(size_t)(cy + 1) * W + cx] = 1;            // Hz(x, y+1)
    }
}

static inline cudaStream_t SS_(void* s) { return reinterpret_cast<cudaStream_t>(s); }

static int grid_for_cells(int64_t n)
{
    const int64_t b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

int launch_shuffle(int n, uint8_t* A, uint8_t* B, uint8_t* F, const DevRng& rng, int* status, uint8_t* canon,
                   uint64_t* launches, void* stream)
{
    const cudaStream_t s = SS_(stream);
    uint8_t *cur = A, *nxt = B;
    const uint32_t tbar = 0x80000000u;   // uniform: horizontal and vertical pairs equally likely
    for (int k = 0; k < n; ++k) {
        const int K = k + 1;
        const dim3 grid((2 * K + 127) / 128, 2 * K);   // x over a row, one block row per cell row
        shuffle_move_kernel<<<grid, 128, 0, s>>>(cur, nxt, n, k);
        shuffle_mark_kernel<<<grid, 128, 0, s>>>(nxt, F, n, K);
        shuffle_create_kernel<<<grid, 128, 0, s>>>(nxt, F, n, K, rng, tbar, status);
        uint8_t* t = cur;
        cur = nxt;
        nxt = t;
    }
    shuffle_canon_kernel<<<grid_for_cells((int64_t)4 * n * n), 256, 0, s>>>(cur, n, canon);
    *launches += (uint64_t)3 * n + 1;
    return (int)cudaGetLastError();
}

}  // namespace tl
