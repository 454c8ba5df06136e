// Domino shuffling: exact uniform random tilings of the Aztec diamond (the
// shuffling algorithms the paper names as an alternative exact sampler,
// Sec. 3; Elkies, Kuperberg, Larsen and Propp).
//
// Cells are unit squares with lower-left corner (x, y), x, y in [-n, n); the
// diamond of order k holds the cells with |x + 1/2| + |y + 1/2| <= k.  A
// cell stores which part of a domino covers it (empty, left / right half of
// a horizontal domino, bottom / top half of a vertical one), one byte per
// cell, rows of S = 2n rounded up to 4 bytes.  In order k a horizontal
// domino with left cell (x, y) goes north if x + y + k is even, else south;
// a vertical one with bottom cell (x, y) goes east if x + y + k is even, else
// west.  One step k -> k + 1 is two data-parallel kernels, each thread
// taking the four cells of one 32-bit word:
//  1. move (gather): every cell of order k + 1 looks at the four cells a
//     domino could arrive from, and takes the part of the one that moves in,
//     unless it is in a bad block (a north-going domino right below a
//     south-going one, or an east-going one right left of a west-going one);
//     all it reads lies in the 3 x 3 cells around it;
//  2. fill: the cells left empty form disjoint 2x2 blocks whose lower-left
//     cells have x + y + k + 1 odd, stacked from the bottom of every run of
//     empty cells in a column.  An empty cell finds its block from its 3 x 3
//     neighbourhood, or where that allows two blocks, from the parity of the
//     run below it and that lower-left parity, and takes its
//     part of the pair the block's Philox draw picks (two horizontal
//     dominoes below 2^31, else two vertical ones).  The result goes to a
//     third buffer, so no thread sees another's output.
#include "tl_device.cuh"

#include <cstdint>

namespace tl {

enum : uint8_t { SH_EMPTY = 0, SH_HL = 1, SH_HR = 2, SH_VB = 3, SH_VT = 4 };

TL_DEV bool in_diamond(int x, int y, int k) { return abs(2 * x + 1) + abs(2 * y + 1) <= 2 * k; }

// Row pitch of the cell buffers in bytes.
TL_DEV int cell_pitch(int n) { return (2 * n + 3) & ~3; }

// Word of this thread: block row blockIdx.y is diamond row y = blockIdx.y - K,
// whose cells are x in [-w, w) with w = K - |y + 1/2| + 1/2; its words run
// from the one holding x = -w to the one holding x = w - 1.  Threads past
// them return false.
TL_DEV bool row_word(int n, int K, int& wi, int& y)
{
    y = (int)blockIdx.y - K;
    const int w = K - (y >= 0 ? y : -y - 1);
    const int wlo = (n - w) >> 2, whi = (n + w + 3) >> 2;
    wi = wlo + (int)(blockIdx.x * blockDim.x + threadIdx.x);
    return wi < whi;
}

// Word wi of buffer row r; 0 (four empty cells) outside the buffer.
TL_DEV uint32_t word_at(const uint8_t* A, int n, int S, int r, int wi)
{
    if (r < 0 || r >= 2 * n || wi < 0 || wi >= S / 4) return 0u;
    return reinterpret_cast<const uint32_t*>(A + (size_t)r * S)[wi];
}

TL_DEV uint8_t byte_of(uint32_t w, int i) { return (uint8_t)(w >> (8 * i)); }

// Cells 4 wi - 1 .. 4 wi + 4 of buffer rows r - 1, r, r + 1: cw[1 + dy][1 + i + dx]
// is the cell (dx, dy) away from cell i of word wi.
TL_DEV void load_window(const uint8_t* A, int n, int S, int r, int wi, uint8_t (&cw)[3][6])
{
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const uint32_t a = word_at(A, n, S, r - 1 + d, wi - 1), b = word_at(A, n, S, r - 1 + d, wi),
                       c = word_at(A, n, S, r - 1 + d, wi + 1);
        cw[d][0] = byte_of(a, 3);
#pragma unroll
        for (int i = 0; i < 4; ++i) cw[d][1 + i] = byte_of(b, i);
        cw[d][5] = byte_of(c, 0);
    }
}

__global__ void shuffle_move_kernel(const uint8_t* __restrict__ A, uint8_t* __restrict__ B, int n, int k)
{
    const int K = k + 1, S = cell_pitch(n);
    int wi, y;
    if (!row_word(n, K, wi, y)) return;
    const int r = y + n;
#ifdef TL_DEBUG
    // the word written: row r of 2n cell rows, bytes 4 wi .. 4 wi + 3 of a pitch-S row
    if (!(TL_IN(r, 2 * n, 501) && TL_IN(4 * wi + 3, S, 502))) return;
#endif
    uint8_t cw[3][6];
    load_window(A, n, S, r, wi, cw);
    uint32_t outw = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int x = 4 * wi + i - n;
        if (!in_diamond(x, y, K)) continue;
        uint8_t out = SH_EMPTY;
        // from below, going north; destroyed if the cell above its left half
        // holds the left half of a south-going one
        uint8_t c = cw[0][1 + i];
        if (c == SH_HL || c == SH_HR) {
            const int ax = c == SH_HL ? x : x - 1;
            if (((ax + y - 1 + k) & 1) == 0 && cw[1][1 + i + (ax - x)] != SH_HL) out = c;
        }
        c = cw[2][1 + i];   // from above, going south
        if (c == SH_HL || c == SH_HR) {
            const int ax = c == SH_HL ? x : x - 1;
            if (((ax + y + 1 + k) & 1) == 1 && cw[1][1 + i + (ax - x)] != SH_HL) out = c;
        }
        c = cw[1][i];   // from the left, going east; destroyed by a west-going one right of it
        if (c == SH_VB || c == SH_VT) {
            const int ay = c == SH_VB ? y : y - 1;
            if (((x - 1 + ay + k) & 1) == 0 && cw[1 + (ay - y)][1 + i] != SH_VB) out = c;
        }
        c = cw[1][2 + i];   // from the right, going west
        if (c == SH_VB || c == SH_VT) {
            const int ay = c == SH_VB ? y : y - 1;
            if (((x + 1 + ay + k) & 1) == 1 && cw[1 + (ay - y)][1 + i] != SH_VB) out = c;
        }
        outw |= (uint32_t)out << (8 * i);
    }
    reinterpret_cast<uint32_t*>(B + (size_t)r * S)[wi] = outw;
}

TL_DEV uint8_t cell_at(const uint8_t* A, int n, int S, int x, int y)
{
    if (x < -n || y < -n || x >= n || y >= n) return SH_EMPTY;
    return A[(size_t)(y + n) * S + (x + n)];
}

// B (after the move, order K) -> C with every hole filled.
// `rngp`: the Philox key and stream, read from device memory so that one
// captured graph of the whole sample serves every seed.
__global__ void shuffle_fill_kernel(const uint8_t* __restrict__ B, uint8_t* __restrict__ C, int n, int K,
                                    const DevRng* __restrict__ rngp, uint32_t tbar, int* __restrict__ status)
{
    const int S = cell_pitch(n);
    int wi, y;
    if (!row_word(n, K, wi, y)) return;
    const int r = y + n;
#ifdef TL_DEBUG
    if (!(TL_IN(r, 2 * n, 503) && TL_IN(4 * wi + 3, S, 504))) return;
#endif
    const uint32_t bw = word_at(B, n, S, r, wi);
    uint32_t outw = bw;
    bool any = false;
#pragma unroll
    for (int i = 0; i < 4; ++i) any |= byte_of(bw, i) == SH_EMPTY && in_diamond(4 * wi + i - n, y, K);
    if (any) {
        const DevRng rng = *rngp;
        uint8_t cw[3][6];
        load_window(B, n, S, r, wi, cw);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int x = 4 * wi + i - n;
            if (cw[1][1 + i] != SH_EMPTY || !in_diamond(x, y, K)) continue;
            // The block holding this cell has its lower-left corner at (x, y)
            // or (x - 1, y - 1) if x + y + K is odd, else at (x - 1, y) or
            // (x, y - 1).  When only one of the two has its other three cells
            // empty, that is the block; otherwise the parity of the run of
            // empty cells below this one in its column decides.
            auto hole = [&](int dx, int dy) {
                return in_diamond(x + dx, y + dy, K) && cw[1 + dy][1 + i + dx] == SH_EMPTY;
            };
            const bool odd = ((x + y + K) & 1) == 1;
            const bool h1 = odd ? hole(1, 0) && hole(0, 1) && hole(1, 1) : hole(-1, 0) && hole(-1, 1) && hole(0, 1);
            const bool h2 = odd ? hole(-1, 0) && hole(0, -1) && hole(-1, -1) : hole(0, -1) && hole(1, -1) && hole(1, 0);
            int bx, by;
            if (h1 != h2) {
                bx = odd ? (h1 ? x : x - 1) : (h1 ? x - 1 : x);
                by = h1 ? y : y - 1;
            } else {
                int below = 0;
                for (int yy = y - 1; yy >= -K && in_diamond(x, yy, K) && cell_at(B, n, S, x, yy) == SH_EMPTY; --yy)
                    ++below;
                by = (below & 1) ? y - 1 : y;
                bx = ((x + by + K) & 1) ? x : x - 1;
            }
            if (x == bx && y == by && (x + 1 >= n || y + 1 >= n || !hole(1, 0) || !hole(0, 1) || !hole(1, 1)))
                atomicExch(status, 1);   // not a 2x2 hole: cannot happen for a valid tiling
            const uint4 o = philox10(((uint32_t)(by + n) << 16) | (uint32_t)(bx + n), (uint32_t)K, 0xFFFE0000u,
                                     rng.stream, rng.k0, rng.k1);
            const uint8_t v = o.x < tbar ? (x > bx ? SH_HR : SH_HL) : (y > by ? SH_VT : SH_VB);
            outw = (outw & ~(0xFFu << (8 * i))) | ((uint32_t)v << (8 * i));
        }
    }
    reinterpret_cast<uint32_t*>(C + (size_t)r * S)[wi] = outw;
}

// Canonical domino state of the order-n diamond (box (2n+1)^2, zeroed):
// a horizontal domino crosses the vertical edge between its cells, a
// vertical one the horizontal edge.
__global__ void shuffle_canon_kernel(const uint8_t* __restrict__ A, int n, uint8_t* __restrict__ canon)
{
    const int S = 2 * n, W = 2 * n + 1, P = cell_pitch(n);
    const int64_t total = (int64_t)S * S;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int cx = (int)(i % S), cy = (int)(i / S);   // cell (cx - n, cy - n)
        const uint8_t v = A[(size_t)cy * P + cx];
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

// A, B, F: three zeroed buffers of 2n rows of (2n rounded up to 4) bytes;
// rng: device copy of the key.  Enqueues 2n + 1 kernels (also under stream
// capture).
int launch_shuffle(int n, uint8_t* A, uint8_t* B, uint8_t* F, const DevRng* rng, int* status, uint8_t* canon,
                   void* stream)
{
    const cudaStream_t s = SS_(stream);
    uint8_t *cur = A, *mid = B, *spare = F;
    const uint32_t tbar = 0x80000000u;   // uniform: horizontal and vertical pairs equally likely
    for (int k = 0; k < n; ++k) {
        const int K = k + 1;
        const int words = ((2 * K + 8) >> 2) + 1;   // words of the widest row, with both ragged ends
        const dim3 grid((words + 127) / 128, 2 * K);   // x over a row's words, one block row per cell row
        shuffle_move_kernel<<<grid, 128, 0, s>>>(cur, mid, n, k);
        shuffle_fill_kernel<<<grid, 128, 0, s>>>(mid, spare, n, K, rng, tbar, status);
        uint8_t* t = cur;
        cur = spare;
        spare = t;
    }
    shuffle_canon_kernel<<<grid_for_cells((int64_t)4 * n * n), 256, 0, s>>>(cur, n, canon);
    return (int)cudaGetLastError();
}

// This file's debug word (failures, then the id, index and bound of the
// first failed check); cudaErrorNotSupported in the normal build.
int dbg_fetch_shuffle(unsigned long long* out, bool clear)
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
