// Split-BF16 block-sparse product on the 5th-generation tensor cores (tcgen05 + TMEM).
//
// C <- beta C + alpha mask_{P_C}(A.B) with every FP64 operand value split into three BF16
// terms x ~ x0 + x1 + x2 (about 26 bits; see split3) and the product formed as the six
// cross products A_p B_q with p + q <= 2, accumulated in FP32 in tensor memory.  Every
// DRAIN chunks (of KSTEPS K steps) the FP32 accumulator is drained into a per-thread
// double-float (hi, lo) sum, so FP32 rounding only acts within a drain period; the result is
// written back in FP64.
//
// Local densification.  9x9 blocks do not fit MMA shapes, so atoms are grouped in space
// (Morton order): an M group holds floor(128/nb) atoms (126 rows for nb = 9), an N group
// floor(64/nb) atoms.  A work tile is a pair (M group g, N group h) that holds at least one
// block of P_C; its K atoms are the atoms k with (i, k) in P_A for some i in g and (k, j)
// in P_B for some j in h.  Absent blocks are zero.  Every C block belongs to exactly one
// tile, so there are no atomics.
//
// K layout (one MMA K step = 16 values = two core-matrix columns of 8).  An atom's orbitals
// are split into a main piece of 8 (orbitals 0-7, nb = 9 only) and a tail of nb - 8 (or
// nb) values.  A main K step holds the main pieces of two K atoms of the tile, paired in
// order, so a tile's main steps follow its own K atom set; a tail K step holds the tails
// of one fixed tail group (16 consecutive atoms in Morton order for nb = 9, 4 for nb = 4),
// taken when the tile has a K atom in the group.  A 9-orbital atom thus costs 8 K values
// plus a sixteenth of a tail step.
//
// Pieces.  Before each product the operands are split and packed into pieces that are
// byte-for-byte shared-memory images in the canonical no-swizzle K-major layout (core
// matrix = 8 rows x 16 bytes; the 8-row groups of one core column adjacent, 128 B apart):
// an A main piece per (M group, atom k) with a block of P_A (3 planes x 128 rows x 8 K,
// 6 KB), an A tail piece per (M group, tail group) with a block (3 planes x 2 columns,
// 12 KB), and B pieces per N group likewise (64 rows: 3 KB and 6 KB).  Shared memory holds
// a K step in an 18 KB slot, so every step costs the same; the descriptors of a main step
// reach its second atom's column through the leading byte offset, those of a tail step
// its second column.  The tile kernel moves each piece with one TMA bulk copy; one thread
// issues the MMAs, eight warps drain the accumulators (bsmm_split_kernel.cuh).  A pieces
// are packed in batches of M groups so that their scratch stays below A_PIECE_CAP bytes.
//
// Bases other than uniform 4 or 9 orbitals (mixed counts, batches of cells) use the same
// pieces and tile kernel with atom groups and tail groups of varying size described by
// tables (bsmm_mixed.cuh).  The emulated-FP64 product (bsmm_emu_kernel.cuh) uses the same
// pieces with eight digit planes instead of three BF16 terms; its K steps come grouped by
// tail group, which is its scale group.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <numeric>

#include "cq_internal.cuh"
#include "emu_digits.cuh"
#include "split3.cuh"

namespace {

constexpr int ST = 320;                      // threads per CTA (10 warps)
constexpr int MT = 128, NT = 64, KCH = 48;   // tile M, N and K chunk
constexpr int KSTEPS = KCH / 16;             // MMA K steps per chunk
constexpr int A_CHUNK = 3 * MT * KCH * 2;   // 36 KB: three planes of 128 rows x 48 K
constexpr int B_CHUNK = 3 * NT * KCH * 2;   // 18 KB
constexpr int STAGE = A_CHUNK + B_CHUNK;    // one shared-memory stage of the split kernel
constexpr int BAR_BYTES = 256;
constexpr int DRAIN = 4;                     // chunks per FP32 accumulation period
constexpr int NACC = 4;                      // FP32 accumulators in tensor memory
constexpr int TMEM_COLS = NACC * NT;
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr size_t A_PIECE_CAP = (size_t)12 << 30;  // scratch bound for one batch of A pieces

// Split-product pieces and the shared-memory slots of one stage (KSTEPS K steps).
constexpr int COLB_A = MT * 16, COLB_B = NT * 16;  // one core column: 2 KB (A), 1 KB (B)
constexpr int A_MAIN = 3 * COLB_A;                 // 6 KB: planes x one column
constexpr int B_MAIN = 3 * COLB_B;                 // 3 KB
constexpr int A_TAIL = 2 * A_MAIN;                 // 12 KB: planes x two columns
constexpr int B_TAIL = 2 * B_MAIN;                 // 6 KB
constexpr int A_SLOT = A_TAIL, B_SLOT = B_TAIL;    // a K step's room in a stage
constexpr int B_SLOTS = KSTEPS * A_SLOT;           // stage offset of the B slots
static_assert(KSTEPS * (A_SLOT + B_SLOT) == STAGE, "stage layout");

// Main and tail widths of an atom's K values, and atoms per tail group.
template <int NB> struct KPieces;
template <> struct KPieces<9> { static constexpr int MAINW = 8, TW = 1, TG = 16; };
template <> struct KPieces<4> { static constexpr int MAINW = 0, TW = 4, TG = 4; };

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of (plane, core column, row) in a piece: planes plane_b apart, core columns
// col_b apart, each column the 8-row groups of its rows 128 B apart
__host__ __device__ __forceinline__ uint32_t piece_off(int plane, int plane_b, int col, int col_b,
                                                       int row)
{
    return (uint32_t)(plane * plane_b + col * col_b + (row >> 3) * 128 + (row & 7) * 16);
}

// shared-memory descriptor, no swizzle: lbo bytes between the two K-adjacent core columns
// of a K step, 128 bytes between 8-row groups
__device__ __forceinline__ uint64_t piece_desc(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // leading (K) byte offset
    d |= (uint64_t)(128 >> 4) << 32;             // stride (M/N) byte offset
    d |= (uint64_t)1 << 46;                      // descriptor version for tcgen05
    return d;                                    // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(MT >> 4) << 24);

// index of block (row, col) in a pattern, or -1
__device__ __forceinline__ int64_t find_block(const int64_t *rp, const int32_t *cl, int row, int col)
{
    int64_t lo = rp[row], hi = rp[row + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (cl[mid] < col)
            lo = mid + 1;
        else
            hi = mid;
    }
    return (lo < rp[row + 1] && cl[lo] == col) ? lo : -1;
}

// ---------------------------------------------------------------- plan kernels

// Tile existence: bit (g, h) for every C block (i, j).
__global__ void k_tile_mark(int64_t n_c, const int32_t *c_row, const int32_t *c_col,
                            const int32_t *g_of, const int32_t *h_of, int n_h, uint32_t *bits)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_c) return;
    const int64_t key = (int64_t)g_of[c_row[b]] * n_h + h_of[c_col[b]];
    atomicOr(&bits[key >> 5], 1u << (key & 31));
}

// Scan of a shared-memory bitmap by a 256-thread CTA: COUNT writes the number of set bits,
// FILL writes their indices in ascending order from out + out0.
template <bool FILL>
__device__ void bitmap_emit(const uint32_t *bits, int words, int64_t *count, int64_t out0,
                            int32_t *out)
{
    __shared__ int scan[256];
    const int per = (words + blockDim.x - 1) / blockDim.x;
    const int w0 = threadIdx.x * per, w1 = min(words, w0 + per);
    int mine = 0;
    for (int w = w0; w < w1; ++w) mine += __popc(bits[w]);
    scan[threadIdx.x] = mine;
    __syncthreads();
    for (int o = 1; o < 256; o <<= 1) {
        int v = threadIdx.x >= o ? scan[threadIdx.x - o] : 0;
        __syncthreads();
        scan[threadIdx.x] += v;
        __syncthreads();
    }
    if (!FILL) {
        if (threadIdx.x == blockDim.x - 1) *count = scan[threadIdx.x];
        return;
    }
    int64_t o = out0 + scan[threadIdx.x] - mine;
    for (int w = w0; w < w1; ++w) {
        uint32_t v = bits[w];
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            out[o++] = w * 32 + bit;
        }
    }
}

// Keys of each atom group (one CTA per group): the key (key_of: Morton rank or tail group;
// atoms with a negative key are left out) of every column of a row of the group's atoms in
// pattern (rp, col).
template <bool FILL>
__global__ void __launch_bounds__(256)
k_group_keys(int gsize, const int32_t *atoms, const int64_t *rp, const int32_t *col,
              const int32_t *key_of, int n_keys, int64_t *count, const int64_t *start,
              int32_t *out)
{
    extern __shared__ uint32_t bits[];
    const int words = (n_keys + 31) >> 5;
    for (int w = threadIdx.x; w < words; w += blockDim.x) bits[w] = 0u;
    __syncthreads();
    for (int s = 0; s < gsize; ++s) {
        const int i = atoms[(int64_t)blockIdx.x * gsize + s];
        if (i < 0) continue;
        for (int64_t e = rp[i] + threadIdx.x; e < rp[i + 1]; e += blockDim.x) {
            const int kk = key_of[col[e]];
            if (kk >= 0) atomicOr(&bits[kk >> 5], 1u << (kk & 31));
        }
    }
    __syncthreads();
    bitmap_emit<FILL>(bits, words, count + blockIdx.x, FILL ? start[blockIdx.x] : 0, out);
}

// Keys of each tile (one CTA per tile): the keys of the atoms k reachable from the M group
// through P_A and from the N group through P_B (P_B symmetric: (k, j) in P_B <=> k in row j).
template <bool FILL>
__global__ void __launch_bounds__(256)
k_tile_keys(int n_atoms, const int2 *tiles, int gi, int gj, const int32_t *g_atoms,
             const int32_t *h_atoms, const int64_t *a_rp, const int32_t *a_col,
             const int64_t *b_rp, const int32_t *b_col, const int32_t *key_of, int n_keys,
             int64_t *count, const int64_t *start, int32_t *out)
{
    extern __shared__ uint32_t bm[];
    const int words = (n_atoms + 31) >> 5, kwords = (n_keys + 31) >> 5;
    uint32_t *ba = bm, *bb = bm + words, *bk = bm + 2 * words;
    for (int w = threadIdx.x; w < 2 * words + kwords; w += blockDim.x) bm[w] = 0u;
    __syncthreads();
    const int2 t = tiles[blockIdx.x];
    for (int s = 0; s < gi; ++s) {
        const int i = g_atoms[(int64_t)t.x * gi + s];
        if (i < 0) continue;
        for (int64_t e = a_rp[i] + threadIdx.x; e < a_rp[i + 1]; e += blockDim.x)
            atomicOr(&ba[a_col[e] >> 5], 1u << (a_col[e] & 31));
    }
    for (int s = 0; s < gj; ++s) {
        const int j = h_atoms[(int64_t)t.y * gj + s];
        if (j < 0) continue;
        for (int64_t e = b_rp[j] + threadIdx.x; e < b_rp[j + 1]; e += blockDim.x)
            atomicOr(&bb[b_col[e] >> 5], 1u << (b_col[e] & 31));
    }
    __syncthreads();
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
        uint32_t v = ba[w] & bb[w];
        while (v) {
            const int bit = __ffs(v) - 1;
            v &= v - 1;
            const int kk = key_of[w * 32 + bit];
            if (kk >= 0) atomicOr(&bk[kk >> 5], 1u << (kk & 31));
        }
    }
    __syncthreads();
    bitmap_emit<FILL>(bk, kwords, count + blockIdx.x, FILL ? start[blockIdx.x] : 0, out);
}

// position of key in the ascending list lst[lo, hi) (the key is present)
__device__ __forceinline__ int64_t list_pos(const int32_t *lst, int64_t lo, int64_t hi, int key)
{
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (lst[mid] < key)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// K-step table of the split product (one CTA per tile): first the main steps, pairing the
// tile's K atoms (Morton ranks, ascending) two by two -- (A main entry, second A main entry
// or -1, B main entry, second B main entry or -1) -- then one tail step per tail group the
// tile touches -- (A tail entry, -1, B tail entry, -1).  Entries index the M group's and
// N group's piece lists.
__global__ void __launch_bounds__(256)
k_tile_steps(const int2 *tiles, const int64_t *ka_start, const int32_t *tile_rank,
             const int64_t *kt_start, const int32_t *tile_tau, const int64_t *step_start,
             const int64_t *gm_ptr, const int32_t *gm_key, const int64_t *hm_ptr,
             const int32_t *hm_key, const int64_t *gt_ptr, const int32_t *gt_key,
             const int64_t *ht_ptr, const int32_t *ht_key, int4 *steps)
{
    const int2 t = tiles[blockIdx.x];
    const int64_t a0 = ka_start[blockIdx.x], na = ka_start[blockIdx.x + 1] - a0;
    const int64_t t0 = kt_start[blockIdx.x], nt = kt_start[blockIdx.x + 1] - t0;
    const int64_t nm = (na + 1) / 2, s0 = step_start[blockIdx.x];
    for (int64_t q = threadIdx.x; q < nm; q += blockDim.x) {
        const int k0 = tile_rank[a0 + 2 * q];
        const int k1 = 2 * q + 1 < na ? tile_rank[a0 + 2 * q + 1] : -1;
        int4 e;
        e.x = (int)list_pos(gm_key, gm_ptr[t.x], gm_ptr[t.x + 1], k0);
        e.y = k1 < 0 ? -1 : (int)list_pos(gm_key, gm_ptr[t.x], gm_ptr[t.x + 1], k1);
        e.z = (int)list_pos(hm_key, hm_ptr[t.y], hm_ptr[t.y + 1], k0);
        e.w = k1 < 0 ? -1 : (int)list_pos(hm_key, hm_ptr[t.y], hm_ptr[t.y + 1], k1);
        steps[s0 + q] = e;
    }
    for (int64_t q = threadIdx.x; q < nt; q += blockDim.x) {
        const int tau = tile_tau[t0 + q];
        steps[s0 + nm + q] = make_int4((int)list_pos(gt_key, gt_ptr[t.x], gt_ptr[t.x + 1], tau), -1,
                                       (int)list_pos(ht_key, ht_ptr[t.y], ht_ptr[t.y + 1], tau), -1);
    }
}

// C block of every (M slot, N slot) pair of each tile: index into P_C or -1, so that the
// epilogue needs one independent load per block instead of a binary search.
__global__ void __launch_bounds__(256)
k_tile_cidx(const int2 *tiles, int gi, int gj, const int32_t *g_atoms, const int32_t *h_atoms,
            const int64_t *c_rp, const int32_t *c_col, int32_t *cidx)
{
    const int2 t = tiles[blockIdx.x];
    for (int e = threadIdx.x; e < gi * gj; e += blockDim.x) {
        const int si = e / gj, sj = e % gj;
        const int i = g_atoms[(int64_t)t.x * gi + si], j = h_atoms[(int64_t)t.y * gj + sj];
        cidx[(int64_t)blockIdx.x * gi * gj + e] =
            (i >= 0 && j >= 0) ? (int32_t)find_block(c_rp, c_col, i, j) : -1;
    }
}

// ---------------------------------------------------------------- piece packing

__device__ __forceinline__ uint32_t pack_bf16x2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// Three BF16 planes of eight values x[0..7] (split3), stored as one 16-byte core-matrix
// row per plane at offsets off + plane * plane_b.
__device__ __forceinline__ void put_row3(uint8_t *dst, uint32_t off, int plane_b,
                                         const double (&x)[8])
{
    __nv_bfloat16 v[3][8];
#pragma unroll
    for (int m = 0; m < 8; ++m) split3(x[m], v[0][m], v[1][m], v[2][m]);
#pragma unroll
    for (int pl = 0; pl < 3; ++pl) {
        uint4 w;
        w.x = pack_bf16x2(v[pl][0], v[pl][1]);
        w.y = pack_bf16x2(v[pl][2], v[pl][3]);
        w.z = pack_bf16x2(v[pl][4], v[pl][5]);
        w.w = pack_bf16x2(v[pl][6], v[pl][7]);
        *reinterpret_cast<uint4 *>(dst + off + pl * plane_b) = w;
    }
}

// Block index of every (slot, key atom) pair of every piece entry (one CTA per entry):
// A side (LEFT): block (i_slot, k) of P_A; B side: block (k, j_slot) of P_B, found as
// block (j, k) of row j and its transpose.  -1 where the pattern has no block.  Patterns
// do not change between products, so the table is built once per pattern triple.
template <bool LEFT>
__global__ void __launch_bounds__(256)
k_piece_index(int gsize, int ca, const int32_t *ent_group, const int32_t *ent_key,
              const int32_t *atoms, const int32_t *key_atoms, const int64_t *rp,
              const int32_t *col, const int64_t *tr, int32_t *index)
{
    const int64_t e = blockIdx.x;
    const int grp = ent_group[e], kk = ent_key[e];
    for (int q = threadIdx.x; q < gsize * ca; q += blockDim.x) {
        const int x = atoms[(int64_t)grp * gsize + q / ca], k = key_atoms[(int64_t)kk * ca + q % ca];
        int64_t b = (x >= 0 && k >= 0) ? find_block(rp, col, x, k) : -1;
        if (!LEFT && b >= 0) b = tr[b];
        index[e * gsize * ca + q] = (int32_t)b;
    }
}

// Main pieces of entries [e0, e0 + n) (one thread per (entry, row)), entry = (atom group,
// K atom k), index = its block per slot (k_piece_index with one atom per key).  A side
// (LEFT): row r = (slot r / NB, orbital o), K = orbital m < 8 of k: A_ik[o][m]; B side: row
// r = (slot, orbital o of j), K = m: B_kj[m][o].
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_main(int64_t e0, int64_t n, const int32_t *index, const double *__restrict__ X,
            int stride, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, COLB = LEFT ? COLB_A : COLB_B;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS;
    const int r = (int)(q % ROWS), o = r % NB;
    const int64_t b = r < G * NB ? __ldg(&index[(e0 + el) * G + r / NB]) : -1;
    double x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
        x[m] = b < 0 ? 0.0 : (LEFT ? X[b * stride + o * NB + m] : X[b * stride + m * NB + o]);
    put_row3(pieces + el * (3 * COLB), piece_off(0, COLB, 0, 0, r), COLB, x);
}

// Tail pieces of entries [e0, e0 + n) (one thread per (entry, row)), entry = (atom group,
// tail group), index = its block per (slot, atom u of the tail group).  K position
// u * TW + m (two core columns) = orbital MAINW + m of atom u.
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_tail(int64_t e0, int64_t n, const int32_t *index, const double *__restrict__ X,
            int stride, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, COLB = LEFT ? COLB_A : COLB_B;
    constexpr int MW = KPieces<NB>::MAINW, TW = KPieces<NB>::TW, TG = KPieces<NB>::TG;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS;
    const int r = (int)(q % ROWS), o = r % NB;
    const int32_t *blk = index + ((e0 + el) * G + (r < G * NB ? r / NB : 0)) * TG;
    uint8_t *piece = pieces + el * (6 * COLB);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        double x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int pos = 8 * c + v, u = pos / TW, m = MW + pos % TW;
            const int64_t b = r < G * NB ? __ldg(&blk[u]) : -1;
            x[v] = b < 0 ? 0.0 : (LEFT ? X[b * stride + o * NB + m] : X[b * stride + m * NB + o]);
        }
        put_row3(piece, piece_off(0, 2 * COLB, c, COLB, r), 2 * COLB, x);
    }
}

__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x)
{
    const float s = hi + x;
    const float bp = s - hi;
    const float err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

struct SplitArgs {
    int n_tiles;              // tiles of this launch
    const int64_t *kstart;    // K-step range of each tile (n_tiles + 1, into steps)
    const int32_t *nmain;     // main K steps of each tile (they come first)
    const int4 *steps;        // piece entries of every K step (k_tile_steps)
    const int32_t *cidx;      // C block of each (M slot, N slot) pair of each tile
    const uint8_t *a_main;    // A main pieces of entries [am0, ...)
    int64_t am0;
    const uint8_t *a_tail;    // A tail pieces of entries [at0, ...)
    int64_t at0;
    const uint8_t *b_main;    // all B main pieces
    const uint8_t *b_tail;    // all B tail pieces
    const uint8_t *zero;      // an all-zero A main piece (stands for a missing second atom)
    double *C;
    int c_stride;
    double alpha, beta;
    int32_t *flag;
    long long test_wait_cycles;  // > 0: test mode, the MMA thread's first wait runs out
    // mixed basis only (bsmm_mixed.cuh): tiles of this launch, row tables, C block offsets
    const int2 *tiles;
    const int32_t *g_row, *h_col;
    const int64_t *c_off;
};

#include "bsmm_mixed.cuh"
#include "bsmm_split_kernel.cuh"
#include "bsmm_emu_kernel.cuh"

constexpr int SMEM = NS * STAGE + BAR_BYTES;     // pipeline stages + barriers
constexpr int SMEM_E = NSE * E_STAGE + E_LWORDS + BAR_BYTES;

// ---------------------------------------------------------------- emulated-FP64 plan and packing

// K-step table of the emulated product (one thread per tile; COUNT writes the number of
// steps of each tile, FILL the steps): per tail group the tile touches (ascending), main
// steps pairing the tile's K atoms of that group (Morton ranks, ascending), then the group's
// tail step; meta flags the first and the last (tail) step of each such scale period.
template <bool FILL>
__global__ void __launch_bounds__(128)
k_emu_steps(int n_tiles, int tg, const int2 *tiles, const int64_t *ka_start,
            const int32_t *tile_rank, const int64_t *kt_start, const int32_t *tile_tau,
            const int64_t *gm_ptr, const int32_t *gm_key, const int64_t *hm_ptr,
            const int32_t *hm_key, const int64_t *gt_ptr, const int32_t *gt_key,
            const int64_t *ht_ptr, const int32_t *ht_key, const int64_t *step_start,
            int64_t *count, int4 *steps, uint8_t *meta)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_tiles) return;
    const int2 t = tiles[b];
    const int64_t a0 = ka_start[b], na = ka_start[b + 1] - a0;
    const int64_t t0 = kt_start[b], nt = kt_start[b + 1] - t0;
    int64_t s = FILL ? step_start[b] : 0, p = 0;
    for (int64_t i = 0; i < nt; ++i) {
        const int tau = tile_tau[t0 + i];
        int64_t p2 = p;
        while (p2 < na && tile_rank[a0 + p2] / tg == tau) ++p2;
        for (int64_t q = p; q < p2; q += 2, ++s) {
            if (!FILL) continue;
            const int k0 = tile_rank[a0 + q], k1 = q + 1 < p2 ? tile_rank[a0 + q + 1] : -1;
            int4 e;
            e.x = (int)list_pos(gm_key, gm_ptr[t.x], gm_ptr[t.x + 1], k0);
            e.y = k1 < 0 ? -1 : (int)list_pos(gm_key, gm_ptr[t.x], gm_ptr[t.x + 1], k1);
            e.z = (int)list_pos(hm_key, hm_ptr[t.y], hm_ptr[t.y + 1], k0);
            e.w = k1 < 0 ? -1 : (int)list_pos(hm_key, hm_ptr[t.y], hm_ptr[t.y + 1], k1);
            steps[s] = e;
            meta[s] = q == p ? PERIOD_FIRST : 0;
        }
        if (FILL) {
            steps[s] = make_int4((int)list_pos(gt_key, gt_ptr[t.x], gt_ptr[t.x + 1], tau), -1,
                                 (int)list_pos(ht_key, ht_ptr[t.y], ht_ptr[t.y + 1], tau), -1);
            meta[s] = PERIOD_LAST | (p2 == p ? PERIOD_FIRST : 0);
        }
        ++s;
        p = p2;
    }
    if (!FILL) count[b] = s;
}

// Group exponent of every row of every tail entry (one thread per (entry, row)): the
// largest emu_exponent of the row's values over the blocks of the entry's tail group (all
// orbitals of its atoms).  A side (LEFT): row r = (slot, orbital o), values A_ik[o][m]; B
// side: column r = (slot, orbital o of j), values B_kj[m][o].
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_emu_rowexp(int64_t n, const int32_t *index, const double *__restrict__ X, int stride,
             int16_t *out)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, TG = KPieces<NB>::TG;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t e = q / ROWS;
    const int r = (int)(q % ROWS), o = r % NB;
    int m = EMU_NONE;
    if (r < G * NB) {
        const int32_t *blk = index + (e * G + r / NB) * TG;
        for (int u = 0; u < TG; ++u) {
            const int64_t b = __ldg(&blk[u]);
            if (b < 0) continue;
            for (int k = 0; k < NB; ++k)
                m = max(m, emu_exponent(LEFT ? X[b * stride + o * NB + k] : X[b * stride + k * NB + o]));
        }
    }
    out[q] = (int16_t)m;
}

// Tail entry of the tail group of every main entry (one thread per main entry): the scale of
// a main piece is its group's.
__global__ void k_emu_main_tail(int64_t n, int tg, const int32_t *group, const int32_t *rank,
                                const int64_t *t_ptr, const int32_t *t_key, int32_t *out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int g = group[e];
    out[e] = (int32_t)list_pos(t_key, t_ptr[g], t_ptr[g + 1], rank[e] / tg);
}

// Eight digit planes of n (<= 8) values as eight 16-byte core-matrix rows (one per plane,
// two BF16 per word, values beyond n zero).
__device__ __forceinline__ void emu_rows(const double *x, int n, int E, uint4 (&w)[EMU_P])
{
    uint32_t u[EMU_P][4];
#pragma unroll
    for (int p = 0; p < EMU_P; ++p)
#pragma unroll
        for (int k = 0; k < 4; ++k) u[p][k] = 0u;
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        if (v >= n) break;
        __nv_bfloat16 d[EMU_P];
        emu_digits(x[v], E, d);
#pragma unroll
        for (int p = 0; p < EMU_P; ++p)
            u[p][v >> 1] |= (uint32_t)__bfloat16_as_ushort(d[p]) << (16 * (v & 1));
    }
#pragma unroll
    for (int p = 0; p < EMU_P; ++p) w[p] = make_uint4(u[p][0], u[p][1], u[p][2], u[p][3]);
}

// Emulated main pieces of entries [e0, e0 + n) (one thread per (entry, row)): as
// k_pack_main, eight digit planes of orbitals 0-7 against the row's group exponent.
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_main_emu(int64_t e0, int64_t n, const int32_t *index, const int32_t *main_tail,
                const int16_t *scale, const double *__restrict__ X, int stride, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, COLB = LEFT ? COLB_A : COLB_B;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS, e = e0 + el;
    const int r = (int)(q % ROWS), o = r % NB;
    const bool row = r < G * NB;
    const int64_t b = row ? __ldg(&index[e * G + r / NB]) : -1;
    const int E = row ? (int)scale[(int64_t)main_tail[e] * ROWS + r] : EMU_NONE;
    double x[8];
#pragma unroll
    for (int m = 0; m < 8; ++m)
        x[m] = b < 0 ? 0.0 : (LEFT ? X[b * stride + o * NB + m] : X[b * stride + m * NB + o]);
    uint4 w[EMU_P];
    emu_rows(x, 8, E, w);
    uint8_t *piece = pieces + el * (EMU_P * COLB);
#pragma unroll
    for (int pl = 0; pl < EMU_P; ++pl)
        *reinterpret_cast<uint4 *>(piece + piece_off(pl, COLB, 0, 0, r)) = w[pl];
}

// Emulated tail pieces of entries [e0, e0 + n) (one thread per (entry, row)): as
// k_pack_tail, eight digit planes against the row's group exponent.
template <int NB, bool LEFT>
__global__ void __launch_bounds__(256)
k_pack_tail_emu(int64_t e0, int64_t n, const int32_t *index, const int16_t *scale,
                const double *__restrict__ X, int stride, uint8_t *pieces)
{
    constexpr int ROWS = LEFT ? MT : NT, G = ROWS / NB, COLB = LEFT ? COLB_A : COLB_B;
    constexpr int MW = KPieces<NB>::MAINW, TW = KPieces<NB>::TW, TG = KPieces<NB>::TG;
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * ROWS) return;
    const int64_t el = q / ROWS, e = e0 + el;
    const int r = (int)(q % ROWS), o = r % NB;
    const bool row = r < G * NB;
    const int32_t *blk = index + (e * G + (row ? r / NB : 0)) * TG;
    const int E = row ? (int)scale[e * ROWS + r] : EMU_NONE;
    uint8_t *piece = pieces + el * (2 * EMU_P * COLB);
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        double x[8];
#pragma unroll
        for (int v = 0; v < 8; ++v) {
            const int pos = 8 * c + v, u = pos / TW, m = MW + pos % TW;
            const int64_t b = row ? __ldg(&blk[u]) : -1;
            x[v] = b < 0 ? 0.0 : (LEFT ? X[b * stride + o * NB + m] : X[b * stride + m * NB + o]);
        }
        uint4 w[EMU_P];
        emu_rows(x, 8, E, w);
#pragma unroll
        for (int pl = 0; pl < EMU_P; ++pl)
            *reinterpret_cast<uint4 *>(piece + piece_off(pl, 2 * COLB, c, COLB, r)) = w[pl];
    }
}

// ---------------------------------------------------------------- host side

struct Groups {
    int gi = 0, gj = 0;              // atoms per M and N group
    int n_g = 0, n_h = 0;
    DevBuf g_atoms, h_atoms, g_of, h_of;
    // K atoms by Morton rank, tail groups of tg consecutive ranks
    int tg = 0, n_tau = 0;
    DevBuf rank_atoms, rank_of, tg_atoms, tg_of;
    // mixed basis (bsmm_mixed.cuh): groups of varying slot counts and their row tables,
    // tail groups of varying atom counts and their position maps; rank_of is -1 for atoms
    // without a main piece
    bool mixed = false;
    DevBuf g_row, h_col, tg_map;
};

// Piece entries of one operand kind (A or B, main or tail): per atom group, ascending keys
// (Morton ranks or tail groups); index = block of every (slot, atom of the key) pair.
struct PieceList {
    DevBuf ptr, key, group, index;
    std::vector<int64_t> ptr_host;
    int64_t n() const { return ptr_host.empty() ? 0 : ptr_host.back(); }
};

struct PieceBatch {
    int tile0, tile1;        // tiles [tile0, tile1)
    int64_t am0, am1;        // A main entries [am0, am1)
    int64_t at0, at1;        // A tail entries [at0, at1)
};

// Piece lists of one product (pattern triple), shared by its split and emulated plans.
struct PieceSet {
    PieceList am, at, bm, bt;  // A main, A tail, B main, B tail
    DevBuf zero;               // an all-zero main piece (stands for a missing second atom)
    DevBuf am_tail, bm_tail;   // emulated product: the tail entry of every main entry's group
};

// Plan of one tensor-core product (pattern triple): tiles, K-step table, batches.  Split
// plans take the main steps of a tile first, then its tail steps; emulated plans take the
// steps of one tail group (its scale period) together, its tail step last, and flag the
// first and last step of every period in meta.
struct PiecePlan {
    int n_tiles = 0;
    int64_t n_steps = 0;
    double mma_flops = 0.0;  // tensor-core flops of one product over these tiles
    std::vector<PieceBatch> batches;
    std::vector<int64_t> batch_steps;
    DevBuf tiles, kstart, nmain, steps, meta, cidx;
    std::shared_ptr<PieceSet> ps;
};

// Morton order of the atoms (positions quantised to 1024 per box edge), cell by cell for a
// batch of cells.
std::vector<int32_t> spatial_order(const Geometry &g)
{
    auto spread = [](uint64_t v) {
        uint64_t x = v & 0x3ff;
        x = (x | (x << 16)) & 0x30000ff;
        x = (x | (x << 8)) & 0x300f00f;
        x = (x | (x << 4)) & 0x30c30c3;
        x = (x | (x << 2)) & 0x9249249;
        return x;
    };
    // a batch keeps its cells apart: the cell index leads the key, each cell in its own box
    const bool batch = g.n_cells > 1 && (int)g.cell_start.size() == g.n_cells + 1;
    std::vector<uint64_t> key(g.n_atoms);
    int cell = 0;
    for (int i = 0; i < g.n_atoms; ++i) {
        while (batch && i >= g.cell_start[cell + 1]) ++cell;
        const double *box = batch ? &g.boxes[3 * cell] : g.box;
        uint64_t c[3];
        for (int d = 0; d < 3; ++d) {
            double f = g.pos_host[3 * i + d] / box[d];
            f -= std::floor(f);
            c[d] = (uint64_t)std::min(1023.0, std::max(0.0, f * 1024.0));
        }
        key[i] = ((uint64_t)cell << 30) | spread(c[0]) | (spread(c[1]) << 1) | (spread(c[2]) << 2);
    }
    std::vector<int32_t> order(g.n_atoms);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t x, int32_t y) { return key[x] < key[y]; });
    return order;
}

cq_status upload(cq_ctx *ctx, DevBuf &buf, const void *host, size_t bytes)
{
    cq_status st = cq_alloc(ctx, buf, bytes ? bytes : 4);
    if (st != CQ_OK) return st;
    if (bytes)
        st = cq_check_cuda(ctx, cudaMemcpyAsync(buf.ptr, host, bytes, cudaMemcpyHostToDevice,
                                                ctx->stream), "upload");
    return st;
}

// Groups of a mixed basis (any orbital counts from 1 to 24; bsmm_mixed.cuh): in the
// spatial order, M groups of consecutive atoms filling at most 128 rows and GI_MIX slots, N
// groups 64 rows and GJ_MIX slots, tail groups of at most TG_MIX atoms whose tails fill at
// most 16 K values; no group spans two cells of a batch.
cq_status mixed_groups(cq_ctx *ctx, const Geometry &g, Groups &gr)
{
    const int n = g.n_atoms;
    for (int i = 0; i < n; ++i)
        if (g.nb_host[i] < 1 || g.nb_host[i] > 24)
            return cq_fail(ctx, CQ_ERR_INVALID,
                           "split-BF16 product: atoms need 1 to 24 orbitals");
    const bool batch = g.n_cells > 1 && (int)g.cell_start.size() == g.n_cells + 1;
    auto cell_of = [&](int atom) {
        if (!batch) return 0;
        return (int)(std::upper_bound(g.cell_start.begin(), g.cell_start.end(), atom) -
                     g.cell_start.begin()) - 1;
    };
    auto tw = [&](int atom) { const int b = g.nb_host[atom]; return b >= 8 ? b - 8 : b; };
    std::vector<int32_t> order = spatial_order(g);
    gr.mixed = true;
    gr.gi = GI_MIX;
    gr.gj = GJ_MIX;
    gr.tg = TG_MIX;
    // greedy groups over the order: a new group when the rows (or tail values) would not fit,
    // the slots are full or the cell changes
    auto make = [&](int cap_rows, int cap_slots, std::vector<int32_t> &atoms,
                    std::vector<int32_t> &rows, std::vector<int32_t> &of) {
        of.assign(n, 0);
        int ng = 0, used = 0, slots = 0, cell = -1;
        std::vector<std::vector<int32_t>> grp;
        for (int r = 0; r < n; ++r) {
            const int a = order[r], b = g.nb_host[a], c = cell_of(a);
            if (grp.empty() || used + b > cap_rows || slots == cap_slots || c != cell) {
                grp.emplace_back();
                ++ng;
                used = slots = 0;
                cell = c;
            }
            grp.back().push_back(a);
            used += b;
            ++slots;
            of[a] = ng - 1;
        }
        atoms.assign((size_t)ng * cap_slots, -1);
        rows.assign((size_t)ng * cap_rows, -1);
        for (int q = 0; q < ng; ++q) {
            int row = 0;
            for (int sl = 0; sl < (int)grp[q].size(); ++sl) {
                const int a = grp[q][sl], b = g.nb_host[a];
                atoms[(size_t)q * cap_slots + sl] = a;
                for (int o = 0; o < b; ++o)
                    rows[(size_t)q * cap_rows + row++] = (sl << 16) | (b << 8) | o;
            }
        }
        return ng;
    };
    std::vector<int32_t> ga, gro, gof, ha, hco, hof;
    gr.n_g = make(MT, GI_MIX, ga, gro, gof);
    gr.n_h = make(NT, GJ_MIX, ha, hco, hof);
    // ranks (main pieces for atoms of 8 orbitals or more) and tail groups
    std::vector<int32_t> rof(n), tof(n), ta, tmap;
    {
        int nt = 0, used = 0, cnt = 0, cell = -1;
        std::vector<std::vector<int32_t>> grp;
        for (int r = 0; r < n; ++r) {
            const int a = order[r], w = tw(a), c = cell_of(a);
            rof[a] = g.nb_host[a] >= 8 ? r : -1;
            if (grp.empty() || used + w > 16 || cnt == TG_MIX || c != cell) {
                grp.emplace_back();
                ++nt;
                used = cnt = 0;
                cell = c;
            }
            grp.back().push_back(a);
            used += w;
            ++cnt;
            tof[a] = nt - 1;
        }
        gr.n_tau = nt;
        ta.assign((size_t)nt * TG_MIX, -1);
        tmap.assign((size_t)nt * TG_MIX, -1);
        for (int q = 0; q < nt; ++q) {
            int pos = 0;
            for (int u = 0; u < (int)grp[q].size(); ++u) {
                const int a = grp[q][u], m0 = g.nb_host[a] >= 8 ? 8 : 0;
                ta[(size_t)q * TG_MIX + u] = a;
                for (int m = 0; m < tw(a); ++m)
                    tmap[(size_t)q * TG_MIX + pos++] = (u << 8) | (m0 + m);
            }
        }
    }
    cq_status st;
    if ((st = upload(ctx, gr.g_atoms, ga.data(), 4 * ga.size())) != CQ_OK ||
        (st = upload(ctx, gr.h_atoms, ha.data(), 4 * ha.size())) != CQ_OK ||
        (st = upload(ctx, gr.g_of, gof.data(), 4 * gof.size())) != CQ_OK ||
        (st = upload(ctx, gr.h_of, hof.data(), 4 * hof.size())) != CQ_OK ||
        (st = upload(ctx, gr.g_row, gro.data(), 4 * gro.size())) != CQ_OK ||
        (st = upload(ctx, gr.h_col, hco.data(), 4 * hco.size())) != CQ_OK ||
        (st = upload(ctx, gr.rank_atoms, order.data(), 4 * order.size())) != CQ_OK ||
        (st = upload(ctx, gr.rank_of, rof.data(), 4 * rof.size())) != CQ_OK ||
        (st = upload(ctx, gr.tg_atoms, ta.data(), 4 * ta.size())) != CQ_OK ||
        (st = upload(ctx, gr.tg_of, tof.data(), 4 * tof.size())) != CQ_OK ||
        (st = upload(ctx, gr.tg_map, tmap.data(), 4 * tmap.size())) != CQ_OK)
        return st;
    return cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "groups");
}

cq_status get_groups(cq_ctx *ctx, const cq_pattern *p, Groups **out)
{
    auto key = std::make_tuple(1, p->geo->id, (uint64_t)0, (uint64_t)0);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = static_cast<Groups *>(it->second.get());
        return CQ_OK;
    }
    const Geometry &g = *p->geo;
    auto gr = std::make_shared<Groups>();
    const int nb = g.uniform_nb;
    if (nb != 9 && nb != 4) {
        cq_status st = mixed_groups(ctx, g, *gr);
        if (st != CQ_OK) return st;
        *out = gr.get();
        ctx->aux[key] = gr;
        return CQ_OK;
    }
    gr->gi = MT / nb;
    gr->gj = NT / nb;
    gr->n_g = (g.n_atoms + gr->gi - 1) / gr->gi;
    gr->n_h = (g.n_atoms + gr->gj - 1) / gr->gj;
    gr->tg = nb == 9 ? KPieces<9>::TG : KPieces<4>::TG;
    gr->n_tau = (g.n_atoms + gr->tg - 1) / gr->tg;
    std::vector<int32_t> order = spatial_order(g);
    std::vector<int32_t> ga((size_t)gr->n_g * gr->gi, -1), ha((size_t)gr->n_h * gr->gj, -1),
        ta((size_t)gr->n_tau * gr->tg, -1);
    std::vector<int32_t> gof(g.n_atoms), hof(g.n_atoms), rof(g.n_atoms), tof(g.n_atoms);
    for (int r = 0; r < g.n_atoms; ++r) {
        ga[r] = ha[r] = ta[r] = order[r];
        gof[order[r]] = r / gr->gi;
        hof[order[r]] = r / gr->gj;
        rof[order[r]] = r;
        tof[order[r]] = r / gr->tg;
    }
    cq_status st;
    if ((st = upload(ctx, gr->g_atoms, ga.data(), 4 * ga.size())) != CQ_OK ||
        (st = upload(ctx, gr->h_atoms, ha.data(), 4 * ha.size())) != CQ_OK ||
        (st = upload(ctx, gr->g_of, gof.data(), 4 * gof.size())) != CQ_OK ||
        (st = upload(ctx, gr->h_of, hof.data(), 4 * hof.size())) != CQ_OK ||
        (st = upload(ctx, gr->rank_atoms, order.data(), 4 * order.size())) != CQ_OK ||
        (st = upload(ctx, gr->rank_of, rof.data(), 4 * rof.size())) != CQ_OK ||
        (st = upload(ctx, gr->tg_atoms, ta.data(), 4 * ta.size())) != CQ_OK ||
        (st = upload(ctx, gr->tg_of, tof.data(), 4 * tof.size())) != CQ_OK)
        return st;
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "groups")) != CQ_OK) return st;
    *out = gr.get();
    ctx->aux[key] = gr;
    return CQ_OK;
}

// Key lists of n_groups atom groups in a pattern, key_of mapping an atom to one of n_keys
// keys (its Morton rank or tail group): every key of a column of a row of the
// group's atoms.  ptr (n_groups + 1), keys (ascending per group), group (entry -> group);
// ptr_host receives ptr.
cq_status group_lists(cq_ctx *ctx, int n_groups, int gsize, const int32_t *atoms,
                      const cq_pattern *p, const int32_t *key_of, int n_keys, DevBuf &ptr,
                      DevBuf &keys, DevBuf &group, std::vector<int64_t> &ptr_host)
{
    cudaStream_t s = ctx->stream;
    cq_status st;
    void *vc;
    if ((st = cq_scratch(ctx, "split_cnt", 8 * ((size_t)n_groups + 1), &vc)) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, ptr, 8 * ((size_t)n_groups + 1))) != CQ_OK) return st;
    const size_t shm = 4 * (size_t)((n_keys + 31) / 32);
    cudaFuncSetAttribute(k_group_keys<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_group_keys<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_group_keys<false><<<n_groups, 256, shm, s>>>(gsize, atoms, p->row_ptr.as<int64_t>(),
                                                    p->col.as<int32_t>(), key_of, n_keys,
                                                    (int64_t *)vc, nullptr, nullptr);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)vc, ptr.as<int64_t>(), n_groups)) != CQ_OK) return st;
    ptr_host.assign((size_t)n_groups + 1, 0);
    cudaMemcpyAsync(ptr_host.data(), ptr.ptr, 8 * ptr_host.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "group lists")) != CQ_OK) return st;
    const int64_t n = ptr_host[n_groups];
    if ((st = cq_alloc(ctx, keys, 4 * (size_t)(n + 1))) != CQ_OK) return st;
    k_group_keys<true><<<n_groups, 256, shm, s>>>(gsize, atoms, p->row_ptr.as<int64_t>(),
                                                   p->col.as<int32_t>(), key_of, n_keys, nullptr,
                                                   ptr.as<int64_t>(), keys.as<int32_t>());
    cq_count_launch();
    std::vector<int32_t> grp((size_t)n);
    for (int q = 0; q < n_groups; ++q)
        for (int64_t e = ptr_host[q]; e < ptr_host[q + 1]; ++e) grp[e] = q;
    if ((st = upload(ctx, group, grp.data(), 4 * grp.size())) != CQ_OK) return st;
    return cq_check_cuda(ctx, cudaStreamSynchronize(s), "group lists");
}

// Work tiles of a product, sorted by (g, h): the (M group, N group) pairs that hold a
// block of P_C.
cq_status tile_list(cq_ctx *ctx, const cq_pattern *pC, const Groups *gr, std::vector<int2> &tiles)
{
    cudaStream_t s = ctx->stream;
    cq_status st;
    const int64_t nbits = (int64_t)gr->n_g * gr->n_h;
    const int64_t nwords = (nbits + 31) / 32;
    void *vb;
    if ((st = cq_scratch(ctx, "split_bits", 4 * nwords, &vb)) != CQ_OK) return st;
    cudaMemsetAsync(vb, 0, 4 * nwords, s);
    if (pC->n_blocks > 0) {
        k_tile_mark<<<(unsigned)((pC->n_blocks + 255) / 256), 256, 0, s>>>(
            pC->n_blocks, pC->row.as<int32_t>(), pC->col.as<int32_t>(), gr->g_of.as<int32_t>(),
            gr->h_of.as<int32_t>(), gr->n_h, (uint32_t *)vb);
        cq_count_launch();
    }
    std::vector<uint32_t> bits(nwords);
    cudaMemcpyAsync(bits.data(), vb, 4 * nwords, cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "tile mark")) != CQ_OK) return st;
    tiles.clear();
    for (int64_t b = 0; b < nbits; ++b)
        if (bits[b >> 5] & (1u << (b & 31)))
            tiles.push_back(make_int2((int)(b / gr->n_h), (int)(b % gr->n_h)));
    return CQ_OK;
}

// Piece list of one operand kind: the keys of every atom group (group_lists) and the block
// of every (slot, key atom) pair (k_piece_index); ca atoms per key, key_atoms listing them.
template <bool LEFT>
cq_status piece_list(cq_ctx *ctx, int n_groups, int gsize, const int32_t *atoms,
                     const cq_pattern *p, const int32_t *key_of, int n_keys, int ca,
                     const int32_t *key_atoms, PieceList &pl)
{
    cq_status st = group_lists(ctx, n_groups, gsize, atoms, p, key_of, n_keys, pl.ptr, pl.key,
                               pl.group, pl.ptr_host);
    if (st != CQ_OK) return st;
    const int64_t n = pl.n();
    if ((st = cq_alloc(ctx, pl.index, 4 * ((size_t)n * gsize * ca + 1))) != CQ_OK) return st;
    if (n > 0) {
        k_piece_index<LEFT><<<(unsigned)n, 256, 0, ctx->stream>>>(
            gsize, ca, pl.group.as<int32_t>(), pl.key.as<int32_t>(), atoms, key_atoms,
            p->row_ptr.as<int64_t>(), p->col.as<int32_t>(),
            LEFT ? nullptr : p->transpose.as<int64_t>(), pl.index.as<int32_t>());
        cq_count_launch();
    }
    return cq_check_cuda(ctx, cudaGetLastError(), "piece index");
}

// Keys of every tile (k_tile_keys with key_of: Morton ranks or tail groups): start
// (n_tiles + 1) on the device and the host, keys ascending per tile.
cq_status tile_keys(cq_ctx *ctx, const DevBuf &tiles, int n_tiles, const Groups *gr,
                    const cq_pattern *pA, const cq_pattern *pB, const int32_t *key_of, int n_keys,
                    DevBuf &start, DevBuf &keys, std::vector<int64_t> &start_host)
{
    cudaStream_t s = ctx->stream;
    const int n_atoms = pA->geo->n_atoms;
    const size_t shm = 4 * (size_t)(2 * ((n_atoms + 31) / 32) + (n_keys + 31) / 32);
    if (shm > 200 * 1024) return cq_fail(ctx, CQ_ERR_INVALID, "split product: too many atoms");
    cq_status st;
    void *vc;
    if ((st = cq_scratch(ctx, "split_cnt", 8 * ((size_t)n_tiles + 1), &vc)) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, start, 8 * ((size_t)n_tiles + 1))) != CQ_OK) return st;
    cudaFuncSetAttribute(k_tile_keys<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    cudaFuncSetAttribute(k_tile_keys<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    k_tile_keys<false><<<n_tiles, 256, shm, s>>>(
        n_atoms, tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
        pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), key_of, n_keys, (int64_t *)vc, nullptr,
        nullptr);
    cq_count_launch();
    if ((st = cq_scan_i64(ctx, (int64_t *)vc, start.as<int64_t>(), n_tiles)) != CQ_OK) return st;
    start_host.assign((size_t)n_tiles + 1, 0);
    cudaMemcpyAsync(start_host.data(), start.ptr, 8 * start_host.size(), cudaMemcpyDeviceToHost, s);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "tile keys")) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, keys, 4 * (size_t)(start_host[n_tiles] + 1))) != CQ_OK) return st;
    k_tile_keys<true><<<n_tiles, 256, shm, s>>>(
        n_atoms, tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(),
        pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(), key_of, n_keys, nullptr,
        start.as<int64_t>(), keys.as<int32_t>());
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "tile keys");
}

cq_status get_pieces(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                     const cq_pattern *pC, const Groups *gr, std::shared_ptr<PieceSet> *out)
{
    auto key = std::make_tuple(5, pA->id, pB->id, pC->id);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = std::static_pointer_cast<PieceSet>(it->second);
        return CQ_OK;
    }
    auto ps = std::make_shared<PieceSet>();
    const int n_atoms = pA->geo->n_atoms;
    cq_status st;
    // main pieces per (atom group, K atom) for 9-orbital atoms, tail pieces per (atom
    // group, tail group)
    if (pC->geo->uniform_nb != 4 &&
        ((st = piece_list<true>(ctx, gr->n_g, gr->gi, gr->g_atoms.as<int32_t>(), pA,
                                gr->rank_of.as<int32_t>(), n_atoms, 1,
                                gr->rank_atoms.as<int32_t>(), ps->am)) != CQ_OK ||
         (st = piece_list<false>(ctx, gr->n_h, gr->gj, gr->h_atoms.as<int32_t>(), pB,
                                 gr->rank_of.as<int32_t>(), n_atoms, 1,
                                 gr->rank_atoms.as<int32_t>(), ps->bm)) != CQ_OK))
        return st;
    if ((st = piece_list<true>(ctx, gr->n_g, gr->gi, gr->g_atoms.as<int32_t>(), pA,
                               gr->tg_of.as<int32_t>(), gr->n_tau, gr->tg,
                               gr->tg_atoms.as<int32_t>(), ps->at)) != CQ_OK ||
        (st = piece_list<false>(ctx, gr->n_h, gr->gj, gr->h_atoms.as<int32_t>(), pB,
                                gr->tg_of.as<int32_t>(), gr->n_tau, gr->tg,
                                gr->tg_atoms.as<int32_t>(), ps->bt)) != CQ_OK)
        return st;
    if ((st = cq_alloc(ctx, ps->zero, E_AMAIN)) != CQ_OK) return st;
    cudaMemsetAsync(ps->zero.ptr, 0, E_AMAIN, ctx->stream);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "pieces")) != CQ_OK) return st;
    *out = ps;
    ctx->aux[key] = ps;
    return CQ_OK;
}

// The plan of a product of kind SPLIT_KIND or EMU_KIND; a_main_b / a_tail_b are the bytes of
// one A main / tail piece of that kind (batch sizing).
constexpr int SPLIT_KIND = 3, EMU_KIND = 4;

cq_status get_piece_plan(cq_ctx *ctx, int kind, const cq_pattern *pA, const cq_pattern *pB,
                         const cq_pattern *pC, const Groups *gr, PiecePlan **out)
{
    auto key = std::make_tuple(kind, pA->id, pB->id, pC->id);
    auto it = ctx->aux.find(key);
    if (it != ctx->aux.end()) {
        *out = static_cast<PiecePlan *>(it->second.get());
        return CQ_OK;
    }
    cudaStream_t s = ctx->stream;
    auto pl = std::make_shared<PiecePlan>();
    const bool mains = pC->geo->uniform_nb != 4, emu = kind == EMU_KIND;
    const int64_t a_main_b = emu ? E_AMAIN : A_MAIN, a_tail_b = emu ? E_ATAIL : A_TAIL;
    const int n_atoms = pA->geo->n_atoms;
    cq_status st;
    if ((st = get_pieces(ctx, pA, pB, pC, gr, &pl->ps)) != CQ_OK) return st;
    const PieceSet &ps = *pl->ps;
    std::vector<int2> tiles;
    if ((st = tile_list(ctx, pC, gr, tiles)) != CQ_OK) return st;
    pl->n_tiles = (int)tiles.size();
    if (tiles.empty()) {
        *out = pl.get();
        ctx->aux[key] = pl;
        return CQ_OK;
    }
    // batches of whole M groups (tiles are sorted by g) whose A pieces fit A_PIECE_CAP
    {
        auto nm_of = [&](int g) { return mains ? ps.am.ptr_host[g] : (int64_t)0; };
        auto a_bytes = [&](int g0, int g1) {  // A pieces of M groups [g0, g1]
            return (nm_of(g1 + 1) - nm_of(g0)) * a_main_b +
                   (ps.at.ptr_host[g1 + 1] - ps.at.ptr_host[g0]) * a_tail_b;
        };
        int t0 = 0;
        while (t0 < pl->n_tiles) {
            const int g0 = tiles[t0].x;
            int t1 = t0, g1 = g0;
            while (t1 < pl->n_tiles) {
                const int g = tiles[t1].x;
                if (g != g1) {  // the next M group starts; keep it only if its pieces still fit
                    if (a_bytes(g0, g) > (int64_t)A_PIECE_CAP) break;
                    g1 = g;
                }
                ++t1;
            }
            pl->batches.push_back({t0, t1, nm_of(g0), nm_of(g1 + 1), ps.at.ptr_host[g0],
                                   ps.at.ptr_host[g1 + 1]});
            t0 = t1;
        }
    }
    if ((st = upload(ctx, pl->tiles, tiles.data(), sizeof(int2) * tiles.size())) != CQ_OK) return st;
    // K atoms and tail groups of every tile (temporaries), then the K-step table
    DevBuf ka_start, tile_rank, kt_start, tile_tau, cnt;
    std::vector<int64_t> ka, kt;
    if (mains) {
        if ((st = tile_keys(ctx, pl->tiles, pl->n_tiles, gr, pA, pB, gr->rank_of.as<int32_t>(),
                            n_atoms, ka_start, tile_rank, ka)) != CQ_OK)
            return st;
    } else {
        ka.assign((size_t)pl->n_tiles + 1, 0);
        if ((st = upload(ctx, ka_start, ka.data(), 8 * ka.size())) != CQ_OK ||
            (st = cq_alloc(ctx, tile_rank, 4)) != CQ_OK)
            return st;
    }
    if ((st = tile_keys(ctx, pl->tiles, pl->n_tiles, gr, pA, pB, gr->tg_of.as<int32_t>(),
                        gr->n_tau, kt_start, tile_tau, kt)) != CQ_OK)
        return st;
    std::vector<int64_t> step_start((size_t)pl->n_tiles + 1, 0);
    std::vector<int32_t> nmain((size_t)pl->n_tiles, 0);
    if (!emu) {
        for (int b = 0; b < pl->n_tiles; ++b) {
            const int64_t nm = (ka[b + 1] - ka[b] + 1) / 2, nt = kt[b + 1] - kt[b];
            nmain[b] = (int32_t)nm;
            step_start[b + 1] = step_start[b] + nm + nt;
        }
    } else {  // per tail group: its atoms' pairs, then its tail step
        if ((st = cq_alloc(ctx, cnt, 8 * ((size_t)pl->n_tiles + 1))) != CQ_OK) return st;
        k_emu_steps<false><<<(pl->n_tiles + 127) / 128, 128, 0, s>>>(
            pl->n_tiles, gr->tg, pl->tiles.as<int2>(), ka_start.as<int64_t>(),
            tile_rank.as<int32_t>(), kt_start.as<int64_t>(), tile_tau.as<int32_t>(), nullptr,
            nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
            cnt.as<int64_t>(), nullptr, nullptr);
        cq_count_launch();
        std::vector<int64_t> c((size_t)pl->n_tiles);
        cudaMemcpyAsync(c.data(), cnt.ptr, 8 * c.size(), cudaMemcpyDeviceToHost, s);
        if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "emu steps")) != CQ_OK) return st;
        for (int b = 0; b < pl->n_tiles; ++b) step_start[b + 1] = step_start[b] + c[b];
    }
    pl->n_steps = step_start[pl->n_tiles];
    pl->mma_flops = (double)pl->n_steps * (emu ? E_MMAS : 6) * 2.0 * MT * NT * 16;
    for (const PieceBatch &bt : pl->batches)
        pl->batch_steps.push_back(step_start[bt.tile1] - step_start[bt.tile0]);
    if ((st = upload(ctx, pl->kstart, step_start.data(), 8 * step_start.size())) != CQ_OK ||
        (st = upload(ctx, pl->nmain, nmain.data(), 4 * nmain.size())) != CQ_OK ||
        (st = cq_alloc(ctx, pl->steps, sizeof(int4) * (size_t)(pl->n_steps + 1))) != CQ_OK ||
        (st = cq_alloc(ctx, pl->cidx, 4 * ((size_t)pl->n_tiles * gr->gi * gr->gj + 1))) != CQ_OK)
        return st;
    if (!emu) {
        k_tile_steps<<<pl->n_tiles, 256, 0, s>>>(
            pl->tiles.as<int2>(), ka_start.as<int64_t>(), tile_rank.as<int32_t>(),
            kt_start.as<int64_t>(), tile_tau.as<int32_t>(), pl->kstart.as<int64_t>(),
            ps.am.ptr.as<int64_t>(), ps.am.key.as<int32_t>(), ps.bm.ptr.as<int64_t>(),
            ps.bm.key.as<int32_t>(), ps.at.ptr.as<int64_t>(), ps.at.key.as<int32_t>(),
            ps.bt.ptr.as<int64_t>(), ps.bt.key.as<int32_t>(), pl->steps.as<int4>());
    } else {
        if ((st = cq_alloc(ctx, pl->meta, (size_t)pl->n_steps + 16)) != CQ_OK) return st;
        k_emu_steps<true><<<(pl->n_tiles + 127) / 128, 128, 0, s>>>(
            pl->n_tiles, gr->tg, pl->tiles.as<int2>(), ka_start.as<int64_t>(),
            tile_rank.as<int32_t>(), kt_start.as<int64_t>(), tile_tau.as<int32_t>(),
            ps.am.ptr.as<int64_t>(), ps.am.key.as<int32_t>(), ps.bm.ptr.as<int64_t>(),
            ps.bm.key.as<int32_t>(), ps.at.ptr.as<int64_t>(), ps.at.key.as<int32_t>(),
            ps.bt.ptr.as<int64_t>(), ps.bt.key.as<int32_t>(), pl->kstart.as<int64_t>(), nullptr,
            pl->steps.as<int4>(), pl->meta.as<uint8_t>());
    }
    k_tile_cidx<<<pl->n_tiles, 256, 0, s>>>(
        pl->tiles.as<int2>(), gr->gi, gr->gj, gr->g_atoms.as<int32_t>(),
        gr->h_atoms.as<int32_t>(), pC->row_ptr.as<int64_t>(), pC->col.as<int32_t>(),
        pl->cidx.as<int32_t>());
    cq_count_launch(2);
    if ((st = cq_check_cuda(ctx, cudaGetLastError(), "piece plan")) != CQ_OK) return st;
    // the temporaries are freed on return: let the kernels that read them finish
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(s), "piece plan")) != CQ_OK) return st;
    *out = pl.get();
    ctx->aux[key] = pl;
    return CQ_OK;
}

template <int NB>
cq_status run_split(cq_ctx *ctx, const PiecePlan *pl, const Groups *gr, double alpha,
                    const cq_pattern *pA, const double *A, const cq_pattern *pB,
                    const double *B, double beta, const cq_pattern *pC, double *C, double flops)
{
    cudaStream_t s = ctx->stream;
    const PieceSet &ps = *pl->ps;
    cq_status st;
    size_t am_bytes = 0, at_bytes = 0;
    for (const PieceBatch &b : pl->batches) {
        am_bytes = std::max(am_bytes, (size_t)(b.am1 - b.am0) * A_MAIN);
        at_bytes = std::max(at_bytes, (size_t)(b.at1 - b.at0) * A_TAIL);
    }
    // one spare piece of room at the end of each piece array
    void *vam, *vat, *vbm, *vbt;
    if ((st = cq_scratch(ctx, "split_Am", am_bytes + A_TAIL, &vam)) != CQ_OK ||
        (st = cq_scratch(ctx, "split_At", at_bytes + A_TAIL, &vat)) != CQ_OK ||
        (st = cq_scratch(ctx, "split_Bm", (size_t)ps.bm.n() * B_MAIN + A_TAIL, &vbm)) != CQ_OK ||
        (st = cq_scratch(ctx, "split_Bt", (size_t)ps.bt.n() * B_TAIL + A_TAIL, &vbt)) != CQ_OK)
        return st;
    // the shared-memory limit is a per-device attribute: set it once per device, on the
    // first split product there (which runs eagerly: building its plan synchronises)
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cq_fail(ctx, CQ_ERR_INVALID, "split product: device index");
    if (!attr_set[dev]) {
        if ((st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_split<9>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM), "split attribute")) != CQ_OK ||
            (st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_split<4>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM), "split attribute")) != CQ_OK ||
            (st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_split<0>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM), "split attribute")) != CQ_OK)
            return st;
        attr_set[dev] = true;
    }
    auto blocks = [](int64_t n, int rows) { return (unsigned)((n * rows + 255) / 256); };
    const int32_t *nbd = pA->geo->nb.as<int32_t>();
    // main and tail pieces of entries [e0, e0 + n) of one side (LEFT: A)
    auto pack = [&](bool left, bool main, int64_t e0, int64_t n, const PieceList &pl_,
                    const double *X, const cq_pattern *pX, void *out) {
        if (n <= 0) return;
        const int rows = left ? MT : NT;
        if constexpr (NB > 0) {
            if (left && main)
                k_pack_main<NB, true><<<blocks(n, rows), 256, 0, s>>>(
                    e0, n, pl_.index.as<int32_t>(), X, pX->uniform, (uint8_t *)out);
            else if (left)
                k_pack_tail<NB, true><<<blocks(n, rows), 256, 0, s>>>(
                    e0, n, pl_.index.as<int32_t>(), X, pX->uniform, (uint8_t *)out);
            else if (main)
                k_pack_main<NB, false><<<blocks(n, rows), 256, 0, s>>>(
                    e0, n, pl_.index.as<int32_t>(), X, pX->uniform, (uint8_t *)out);
            else
                k_pack_tail<NB, false><<<blocks(n, rows), 256, 0, s>>>(
                    e0, n, pl_.index.as<int32_t>(), X, pX->uniform, (uint8_t *)out);
        } else {
            const int32_t *tab = left ? gr->g_row.as<int32_t>() : gr->h_col.as<int32_t>();
            const int64_t *off = pX->val_off.as<int64_t>();
            if (main) {
                auto k = left ? k_pack_main_mixed<true> : k_pack_main_mixed<false>;
                k<<<blocks(n, rows), 256, 0, s>>>(e0, n, pl_.index.as<int32_t>(),
                                                  pl_.group.as<int32_t>(), pl_.key.as<int32_t>(),
                                                  gr->rank_atoms.as<int32_t>(), tab, nbd, off, X,
                                                  (uint8_t *)out);
            } else {
                auto k = left ? k_pack_tail_mixed<true> : k_pack_tail_mixed<false>;
                k<<<blocks(n, rows), 256, 0, s>>>(e0, n, pl_.index.as<int32_t>(),
                                                  pl_.group.as<int32_t>(), pl_.key.as<int32_t>(),
                                                  gr->tg_atoms.as<int32_t>(),
                                                  gr->tg_map.as<int32_t>(), tab, nbd, off, X,
                                                  (uint8_t *)out);
            }
        }
        cq_count_launch();
    };
    pack(false, true, 0, ps.bm.n(), ps.bm, B, pB, vbm);
    pack(false, false, 0, ps.bt.n(), ps.bt, B, pB, vbt);
    for (size_t q = 0; q < pl->batches.size(); ++q) {
        const PieceBatch &b = pl->batches[q];
        pack(true, true, b.am0, b.am1 - b.am0, ps.am, A, pA, vam);
        pack(true, false, b.at0, b.at1 - b.at0, ps.at, A, pA, vat);
        SplitArgs a;
        a.n_tiles = b.tile1 - b.tile0;
        a.kstart = pl->kstart.as<int64_t>() + b.tile0;
        a.nmain = pl->nmain.as<int32_t>() + b.tile0;
        a.steps = pl->steps.as<int4>();
        a.cidx = pl->cidx.as<int32_t>() + (int64_t)b.tile0 * gr->gi * gr->gj;
        a.a_main = (const uint8_t *)vam;
        a.am0 = b.am0;
        a.a_tail = (const uint8_t *)vat;
        a.at0 = b.at0;
        a.b_main = (const uint8_t *)vbm;
        a.b_tail = (const uint8_t *)vbt;
        a.zero = ps.zero.as<uint8_t>();
        a.C = C;
        a.c_stride = pC->uniform;
        a.alpha = alpha;
        a.beta = beta;
        a.flag = ctx->flag.as<int32_t>();
        a.test_wait_cycles = ctx->test_wait_cycles;
        a.tiles = pl->tiles.as<int2>() + b.tile0;
        a.g_row = gr->g_row.as<int32_t>();
        a.h_col = gr->h_col.as<int32_t>();
        a.c_off = pC->val_off.as<int64_t>();
        // this launch's share of the product's useful and tensor-core flops
        const double share =
            pl->n_steps > 0 ? (double)pl->batch_steps[q] / (double)pl->n_steps : 0.0;
        const int grid = std::min(a.n_tiles, ctx->num_sms);
        cq_timing_begin(ctx, flops * share, pl->mma_flops * share);
        k_bsmm_split<NB><<<grid, ST, SMEM, s>>>(a);
        cq_timing_end(ctx);
        cq_count_launch();
        if ((st = cq_check_cuda(ctx, cudaGetLastError(), "bsmm_split")) != CQ_OK) return st;
    }
    return CQ_OK;
}

template <int NB>
cq_status run_emu(cq_ctx *ctx, PiecePlan *pl, const Groups *gr, double alpha,
                  const cq_pattern *pA, const double *A, const cq_pattern *pB, const double *B,
                  double beta, const cq_pattern *pC, double *C, double flops)
{
    cudaStream_t s = ctx->stream;
    PieceSet &ps = *pl->ps;
    cq_status st;
    auto blocks = [](int64_t n, int rows) { return (unsigned)((n * rows + 255) / 256); };
    // tail entry of every main entry (once per piece set)
    if (ps.am.n() > 0 && !ps.am_tail.ptr) {
        if ((st = cq_alloc(ctx, ps.am_tail, 4 * (size_t)ps.am.n())) != CQ_OK ||
            (st = cq_alloc(ctx, ps.bm_tail, 4 * (size_t)ps.bm.n() + 4)) != CQ_OK)
            return st;
        k_emu_main_tail<<<blocks(ps.am.n(), 1), 256, 0, s>>>(
            ps.am.n(), gr->tg, ps.am.group.as<int32_t>(), ps.am.key.as<int32_t>(),
            ps.at.ptr.as<int64_t>(), ps.at.key.as<int32_t>(), ps.am_tail.as<int32_t>());
        cq_count_launch();
        if (ps.bm.n() > 0) {
            k_emu_main_tail<<<blocks(ps.bm.n(), 1), 256, 0, s>>>(
                ps.bm.n(), gr->tg, ps.bm.group.as<int32_t>(), ps.bm.key.as<int32_t>(),
                ps.bt.ptr.as<int64_t>(), ps.bt.key.as<int32_t>(), ps.bm_tail.as<int32_t>());
            cq_count_launch();
        }
    }
    size_t am_bytes = 0, at_bytes = 0;
    for (const PieceBatch &b : pl->batches) {
        am_bytes = std::max(am_bytes, (size_t)(b.am1 - b.am0) * E_AMAIN);
        at_bytes = std::max(at_bytes, (size_t)(b.at1 - b.at0) * E_ATAIL);
    }
    // one spare piece of room at the end of each piece array
    void *vam, *vat, *vbm, *vbt, *sa, *sb;
    if ((st = cq_scratch(ctx, "emu_Am", am_bytes + E_ATAIL, &vam)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_At", at_bytes + E_ATAIL, &vat)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_Bm", (size_t)ps.bm.n() * E_BMAIN + E_ATAIL, &vbm)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_Bt", (size_t)ps.bt.n() * E_BTAIL + E_ATAIL, &vbt)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_sa", 2 * (size_t)ps.at.n() * MT + 16, &sa)) != CQ_OK ||
        (st = cq_scratch(ctx, "emu_sb", 2 * (size_t)ps.bt.n() * NT + 16, &sb)) != CQ_OK)
        return st;
    // the shared-memory limit is a per-device attribute: set it once per device
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cq_fail(ctx, CQ_ERR_INVALID, "emulated product: device index");
    if (!attr_set[dev]) {
        if ((st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_emu<9>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM_E), "emu attribute")) != CQ_OK ||
            (st = cq_check_cuda(ctx, cudaFuncSetAttribute(k_bsmm_emu<4>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                          SMEM_E), "emu attribute")) != CQ_OK)
            return st;
        attr_set[dev] = true;
    }
    // group exponents (every tail entry: the groups of one M group may fall in different
    // packing batches), then the digit planes of B and of each batch of A
    if (ps.bt.n() > 0) {
        k_emu_rowexp<NB, false><<<blocks(ps.bt.n(), NT), 256, 0, s>>>(
            ps.bt.n(), ps.bt.index.as<int32_t>(), B, pB->uniform, (int16_t *)sb);
        k_pack_tail_emu<NB, false><<<blocks(ps.bt.n(), NT), 256, 0, s>>>(
            0, ps.bt.n(), ps.bt.index.as<int32_t>(), (const int16_t *)sb, B, pB->uniform,
            (uint8_t *)vbt);
        cq_count_launch(2);
    }
    if (ps.bm.n() > 0) {
        k_pack_main_emu<NB, false><<<blocks(ps.bm.n(), NT), 256, 0, s>>>(
            0, ps.bm.n(), ps.bm.index.as<int32_t>(), ps.bm_tail.as<int32_t>(),
            (const int16_t *)sb, B, pB->uniform, (uint8_t *)vbm);
        cq_count_launch();
    }
    if (ps.at.n() > 0) {
        k_emu_rowexp<NB, true><<<blocks(ps.at.n(), MT), 256, 0, s>>>(
            ps.at.n(), ps.at.index.as<int32_t>(), A, pA->uniform, (int16_t *)sa);
        cq_count_launch();
    }
    for (size_t q = 0; q < pl->batches.size(); ++q) {
        const PieceBatch &b = pl->batches[q];
        if (b.am1 > b.am0) {
            k_pack_main_emu<NB, true><<<blocks(b.am1 - b.am0, MT), 256, 0, s>>>(
                b.am0, b.am1 - b.am0, ps.am.index.as<int32_t>(), ps.am_tail.as<int32_t>(),
                (const int16_t *)sa, A, pA->uniform, (uint8_t *)vam);
            cq_count_launch();
        }
        if (b.at1 > b.at0) {
            k_pack_tail_emu<NB, true><<<blocks(b.at1 - b.at0, MT), 256, 0, s>>>(
                b.at0, b.at1 - b.at0, ps.at.index.as<int32_t>(), (const int16_t *)sa, A,
                pA->uniform, (uint8_t *)vat);
            cq_count_launch();
        }
        EmuArgs a;
        a.n_tiles = b.tile1 - b.tile0;
        a.kstart = pl->kstart.as<int64_t>() + b.tile0;
        a.steps = pl->steps.as<int4>();
        a.meta = pl->meta.as<uint8_t>();
        a.cidx = pl->cidx.as<int32_t>() + (int64_t)b.tile0 * gr->gi * gr->gj;
        a.a_main = (const uint8_t *)vam;
        a.am0 = b.am0;
        a.a_tail = (const uint8_t *)vat;
        a.at0 = b.at0;
        a.b_main = (const uint8_t *)vbm;
        a.b_tail = (const uint8_t *)vbt;
        a.zero = ps.zero.as<uint8_t>();
        a.scale_a = (const int16_t *)sa;
        a.scale_b = (const int16_t *)sb;
        a.C = C;
        a.c_stride = pC->uniform;
        a.alpha = alpha;
        a.beta = beta;
        a.flag = ctx->flag.as<int32_t>();
        const double share =
            pl->n_steps > 0 ? (double)pl->batch_steps[q] / (double)pl->n_steps : 0.0;
        const int grid = std::min(a.n_tiles, ctx->num_sms);
        cq_timing_begin(ctx, flops * share, pl->mma_flops * share);
        k_bsmm_emu<NB><<<grid, ST, SMEM_E, s>>>(a);
        cq_timing_end(ctx);
        cq_count_launch();
        if ((st = cq_check_cuda(ctx, cudaGetLastError(), "bsmm_emu")) != CQ_OK) return st;
    }
    return CQ_OK;
}

}  // namespace

cq_status cq_bsmm_emu(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                      const double *A, const cq_pattern *pB, const double *B, double beta,
                      const cq_pattern *pC, double *C)
{
    const int nb = pC->geo->uniform_nb;
    if (nb != 9 && nb != 4)
        return cq_fail(ctx, CQ_ERR_INVALID,
                       "emulated-FP64 product: needs a uniform basis of 4 or 9 orbitals per atom");
    if (pC->n_blocks == 0) return CQ_OK;
    Groups *gr;
    PiecePlan *pl;
    cq_status st = get_groups(ctx, pC, &gr);
    if (st != CQ_OK) return st;
    if ((st = get_piece_plan(ctx, EMU_KIND, pA, pB, pC, gr, &pl)) != CQ_OK) return st;
    if (pl->n_tiles == 0) return CQ_OK;
    return nb == 9 ? run_emu<9>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops)
                   : run_emu<4>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops);
}

cq_status cq_bsmm_split(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                        const double *A, const cq_pattern *pB, const double *B, double beta,
                        const cq_pattern *pC, double *C)
{
    const int nb = pC->geo->uniform_nb;  // 4 and 9: uniform kernels; otherwise the mixed path
    if (pC->n_blocks == 0) return CQ_OK;
    Groups *gr;
    PiecePlan *pl;
    cq_status st = get_groups(ctx, pC, &gr);
    if (st != CQ_OK) return st;
    if ((st = get_piece_plan(ctx, SPLIT_KIND, pA, pB, pC, gr, &pl)) != CQ_OK) return st;
    if (pl->n_tiles == 0) return CQ_OK;
    if (nb == 9) return run_split<9>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops);
    if (nb == 4) return run_split<4>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops);
    return run_split<0>(ctx, pl, gr, alpha, pA, A, pB, B, beta, pC, C, tl->flops);
}
