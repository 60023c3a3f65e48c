/*
 * cq.h -- C ABI of the GB300 block-sparse linear-scaling solver library (libcq.so).
 *
 * The paper (Bowler, Miyazaki, Nakata, Truflandier, "The CONQUEST code: large scale and
 * linear scaling DFT") states the method in words: a linear-scaling ground-state solver
 * that keeps its matrices sparse so every operation stays local (Background), minimises
 * the energy over the density matrix and inverts the overlap, both in linear-scaling time
 * (Development Priorities), and names the sparse matrix product as the first kernel to move
 * to GPUs (Meeting the Exascale Challenges).  The calls below expose exactly that hot
 * path: range-cutoff patterns, the atom-blocked product kept on C's pattern, traces, the
 * Hotelling inversion step T <- 2T - TST, the Li-Nunes-Vanderbilt (LNV) density-matrix step
 * with K = 3LSL - 2LSLSL, its Palser-Manolopoulos start and McWeeny purification.
 *
 * Conventions shared by every call
 * --------------------------------
 *  Units: bohr, hartree.  Matrices are Gamma-point, atom-blocked: block (i, j) is an
 *  nb[i] x nb[j] row-major FP64 array.  A pattern P_R holds every ordered pair (i, j) whose
 *  minimum-image distance in the orthorhombic box is below R (i == j always included), so
 *  every pattern is symmetric.  Its blocks are ordered by atom row i, then column j
 *  ascending; block b starts at val_off[b] doubles into the value array, and every block
 *  starts on a 16-byte boundary (its size is padded to an even number of doubles; padding
 *  values are unspecified).  n_values is the length of a value array on the pattern.
 *
 *  Memory: every `const double*` / `double*` value array and every `*_dev` argument is
 *  caller-owned device memory on the context's device, contiguous, never freed or kept by
 *  the library past the call.  Host pointers are marked `_host`.  Opaque objects
 *  (cq_ctx, cq_pattern, cq_lnv) are owned by the library and released by their destroy
 *  call.  Scratch (task lists, intermediate products) belongs to the context or the LNV
 *  object; nothing returned needs to be freed by the caller.
 *
 *  Devices: calls on a context expect its device to be the current CUDA device (the one
 *  passed to cq_ctx_create), as with other CUDA libraries; the library does not switch.
 *
 *  Streams: all device work is enqueued on the stream given to cq_ctx_create, in order.
 *  Calls returning host scalars synchronise that stream.
 *
 *  Errors: every call returns a cq_status and never aborts or traps; cq_last_error gives
 *  the context's last message.  Asynchronous CUDA failures surface as CQ_ERR_CUDA at the
 *  next synchronising call.
 */
#ifndef CQ_H
#define CQ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CQ_OK = 0,
    CQ_ERR_INVALID = 1,       /* bad argument (null pointer, size, range, precision)      */
    CQ_ERR_PATTERN = 2,       /* patterns of different atoms/basis, or block not in pattern */
    CQ_ERR_NOMEM = 3,         /* device allocation failed (or the context's limit reached) */
    CQ_ERR_CUDA = 4,          /* a CUDA runtime call or kernel failed                     */
    CQ_ERR_NUMERIC = 5,       /* NaN or Inf in a scalar result                            */
    CQ_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out                       */
    CQ_ERR_NOT_CONVERGED = 7  /* an iteration hit its limit                               */
} cq_status;

typedef enum {
    CQ_FP64 = 0,          /* block products on FP64 FMAs                                   */
    CQ_SPLIT_BF16X3 = 1,  /* products as 3-term split-BF16 on tensor cores, FP32 accumulate */
    CQ_FP64_EMU = 2       /* FP64-accurate products on the BF16 tensor cores: 8 digit planes
                             per value, exact level sums, three-float drains (see cq_bsmm) */
} cq_precision;

typedef struct cq_ctx cq_ctx;
typedef struct cq_pattern cq_pattern;
typedef struct cq_lnv cq_lnv;

/* ---------------------------------------------------------------- context */

/* Create a context on `device`, enqueuing on `cuda_stream` (a cudaStream_t, borrowed, may
 * be NULL for the legacy default stream).  *out receives the context. */
cq_status cq_ctx_create(int device, void *cuda_stream, cq_ctx **out);
void cq_ctx_destroy(cq_ctx *ctx);
/* Last error message of the context (never NULL; "" when none). */
const char *cq_last_error(const cq_ctx *ctx);
/* Synchronise the context's stream and report any pending asynchronous error. */
cq_status cq_ctx_sync(cq_ctx *ctx);
/* Cap the context's own device allocations at `bytes` (0 = no cap); an allocation beyond it
 * fails with CQ_ERR_NOMEM, as a real out-of-memory would.  Used to test that path. */
cq_status cq_ctx_set_mem_limit(cq_ctx *ctx, int64_t bytes);
/* Free everything the context caches to speed up later calls: (i, k, j) task lists, block
 * maps, tensor-core tile plans and scratch buffers (patterns, values and LNV objects are
 * untouched).  Later calls rebuild what they need, and LNV graph phases are captured anew.
 * For working sets near the size of HBM: e.g. after the FP64 set-up of a large cell
 * (Hotelling inverse, PM start), before tensor-core LNV steps that never use the FP64 task
 * lists.  Synchronises; refused inside a graph capture. */
cq_status cq_ctx_release_cache(cq_ctx *ctx);
/* Bytes of device scratch the context currently holds. */
int64_t cq_ctx_mem_used(const cq_ctx *ctx);
/* Turn on (1) or off (0) CUDA-event timing of every block-product kernel launch on the
 * context's stream (for roofline reporting; off by default). */
cq_status cq_ctx_set_timing(cq_ctx *ctx, int on);
/* Totals since the last call (then reset): product kernel launches, their summed device
 * time in ms, their useful flops (sum 2 n_i n_k n_j) and the tensor-core flops the split and
 * emulated products issued, padding included (0 for FP64 products).  Synchronises. */
cq_status cq_ctx_kernel_stats(cq_ctx *ctx, int64_t *launches_host, double *ms_host,
                              double *flops_host, double *mma_flops_host);
/* Autotuner (off by default): on the first FP64 product of each (P_A, P_B, P_C) triple, time
 * every lane split of the FP64 kernel (1..32 lanes per C row) on the real operands into
 * scratch and keep the fastest for that triple.  Synchronises on that first use only. */
cq_status cq_ctx_set_autotune(cq_ctx *ctx, int on);
/* CUDA graphs (off by default): LNV evaluation phases (trial point, electron-number half,
 * energy half: their products, traces and gradients) run eagerly once, are captured on
 * their second use and replayed afterwards, with identical results.  Needs a context on a
 * created stream (the legacy default stream cannot be captured): CQ_ERR_INVALID otherwise. */
cq_status cq_ctx_set_graphs(cq_ctx *ctx, int on);
/* Test hook for the error path of the tensor-core waits (0 = off, the default).  With
 * cycles > 0 every later split-BF16 product kernel makes its first wait on a barrier that
 * nothing completes, gives up after `cycles` clock cycles (at most 1e8) and takes the same
 * path as a real timeout: the CTA stops issuing, retires the copies it issued (with the
 * normal bounded wait), frees its tensor memory and returns; the next synchronising call
 * returns CQ_ERR_TIMEOUT and C is incomplete.  Nothing waits without a bound. */
cq_status cq_ctx_set_test_wait(cq_ctx *ctx, int64_t cycles);
/* Lanes per C row the FP64 product of this triple uses, and whether the autotuner chose it. */
cq_status cq_bsmm_config(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                         const cq_pattern *pC, int32_t *lane_split_host, int32_t *tuned_host);
/* Measure the device's FP64 throughput (flop/s, an FMA counted as 2): the better of two
 * register-resident probes filling every SM, a chain of independent FP64 FMAs and a chain of
 * FP64 tensor-core MMAs (m8n8k4), each timed over five launches after a warm-up launch.  The
 * FP64 roofline denominator.  Synchronises the context stream; takes about a second. */
cq_status cq_peak_fp64(cq_ctx *ctx, double *flops_per_s_host);
/* Number of CUDA kernels this library has launched in the process. */
int64_t cq_kernel_launches(void);

/* ---------------------------------------------------------------- patterns */

/*
 * Build P_range = {(i, j) : d_min(i, j) < range} over n_atoms atoms (Background: locality
 * through range-cutoff sparse storage).  pos_dev: n_atoms x 3 FP64 positions; box_host:
 * the three box lengths; nb_dev: orbitals per atom (1..16).  The squared distance is
 * evaluated in FP64 as ((dx*dx + dy*dy) + dz*dz) with d = (x_j - x_i) - box*rint((x_j -
 * x_i)/box), without FMA contraction.  The pattern keeps its own copy of the geometry.
 */
cq_status cq_pattern_build(cq_ctx *ctx, int32_t n_atoms, const double *pos_dev,
                           const double *box_host, const int32_t *nb_dev, double range,
                           cq_pattern **out);
/*
 * Batch of n_cells independent periodic cells (up to 1024) as one pattern: the atoms of
 * cell c are cell_start_host[c] .. cell_start_host[c+1]-1 (cell_start_host[0] = 0, no empty
 * cell), cell c has box boxes_host[3c..3c+2] and range ranges_host[c]; pairs never cross
 * cells.  Products over a batch pattern compute every cell in one launch; traces, dots and
 * the LNV / Hotelling / PM scalars are kept per cell (the *_cells entry points).  Blocks of
 * a cell are contiguous in the pattern (its rows are).
 */
cq_status cq_pattern_build_batch(cq_ctx *ctx, int32_t n_cells, const int32_t *cell_start_host,
                                 const double *pos_dev, const double *boxes_host,
                                 const int32_t *nb_dev, const double *ranges_host,
                                 cq_pattern **out);
/* Number of cells of a pattern (1 unless built by cq_pattern_build_batch). */
int32_t cq_pattern_cells(const cq_pattern *p);
/* Sizes of a pattern: number of blocks and length of a value array. */
cq_status cq_pattern_info(const cq_pattern *p, int64_t *n_blocks, int64_t *n_values);
/* Copy the pattern's index arrays into caller buffers (any may be NULL): row_ptr
 * (n_atoms + 1, int64), col (n_blocks, int32), val_off (n_blocks, int64, in doubles),
 * transpose (n_blocks, int64: index of block (j, i)). */
cq_status cq_pattern_export(cq_ctx *ctx, const cq_pattern *p, int64_t *row_ptr_dev,
                            int32_t *col_dev, int64_t *val_off_dev, int64_t *transpose_dev);
void cq_pattern_destroy(cq_pattern *p);

/*
 * Fill a value array on p from a coordinate list of n_pairs blocks: pair b is block
 * (pair_i[b], pair_j[b]) with nb[i]*nb[j] row-major values at pair_values + pair_off[b].
 * Blocks not listed are zero.  A listed block outside p gives CQ_ERR_PATTERN (detected on
 * the device, reported by this call, which synchronises).
 */
cq_status cq_pattern_scatter(cq_ctx *ctx, const cq_pattern *p, int64_t n_pairs,
                             const int32_t *pair_i_dev, const int32_t *pair_j_dev,
                             const int64_t *pair_off_dev, const double *pair_values_dev,
                             double *out);

/* ---------------------------------------------------------------- products and traces */

/*
 * C <- beta*C + alpha*mask_{P_C}(A.B): for every block (i, j) of P_C,
 * C_ij = beta*C_ij + alpha * sum_k A_ik B_kj over the k with (i, k) in P_A and (k, j) in
 * P_B (the sparse matrix multiplication of the paper's Background and Exascale sections).
 * With beta == 0 the old C is not read.  The (i, k, j) task list of each (P_A, P_B, P_C)
 * triple is built on the device on first use and cached in the context.  C must not alias
 * A or B.  prec selects FP64 FMAs or one of the tensor-core products.  The split product
 * takes uniform bases of 4 or 9 orbitals per atom on its uniform kernels and every other
 * basis a pattern can hold (1 to 16 orbitals per atom, mixed counts and batches of cells
 * included) on its mixed path.  It packs both operands into context-owned scratch
 * before every call (up to about 2x the FP64 size of the operands, the A side in batches of
 * at most 12 GB), and its accuracy is FP32-class:
 * about 1e-7 relative per block, with FP32 partial sums drained to double-float.  Each value
 * is split to about 2^-27 relative for 2^-74 <= |x| < (2 - 2^-8) 2^127 (coarser below,
 * zero under 2^-126); larger values, infinities and NaNs give NaN in every C value they
 * reach, so the next trace reports CQ_ERR_NUMERIC as with FP64.
 *
 * CQ_FP64_EMU gives FP64-class products on the BF16 tensor cores (Ozaki-style slicing; the
 * paper's priorities of GPU products and solver accuracy together, on a GPU whose FP64 pipe
 * is narrow): per scalar row of A and scalar column of B over every sixteen consecutive atoms
 * of K in the spatial (Morton) order (four for a 4-orbital basis) a power-of-two scale 2^E
 * with |x| < 2^E; every value is rounded to the grid
 * 2^(E-63) and cut into eight signed 8-bit digits, each exact in BF16; the 36 digit
 * products of levels p + q <= 7 run on the tensor cores, levels 0-4 summed exactly in FP32
 * within a scale period and levels 5-7 together, and every period drains into a three-float
 * (about 72-bit) sum.  Every value is carried to 2^-64 of its group's largest magnitude,
 * so the error of C_ij stays below about 1e-15 sum_k (Amax ||B_kj|| + ||A_ik|| Bmax) with
 * Amax, Bmax the largest magnitudes of the scale groups the terms fall in.  While the
 * magnitudes inside a group stay within about 2^14 of one another (the smooth decay of the
 * method's matrices) that is the FP64 product bound
 * ||dC_ij|| <= 1e-12 max(||C_ij||, 1e-3 sum_k ||A_ik|| ||B_kj||); terms must lie between
 * about 2^-70 and 2^120 in magnitude (FP32's range holds the drained sums).
 * It needs a uniform basis of 4 or 9 orbitals per atom (else CQ_ERR_INVALID); its packed
 * operands take about 2.7x the split's scratch (eight BF16 planes per value).  Infinities
 * and NaNs poison their scale group: they give NaN in every C value of the rows (of A) or
 * columns (of B) that group reaches.
 *
 * The tensor-core calls are asynchronous on the context stream; if a bounded wait inside a
 * tensor-core kernel (split or emulated) ran out (a copy or MMA completion not seen within
 * about two seconds), the next synchronising call on the context (cq_ctx_sync, a trace, a
 * dot, an LNV or Hotelling step) returns CQ_ERR_TIMEOUT and C is incomplete.
 */
cq_status cq_bsmm(cq_ctx *ctx, double alpha, const cq_pattern *pA, const double *A,
                  const cq_pattern *pB, const double *B, double beta,
                  const cq_pattern *pC, double *C, cq_precision prec);

/* Number of (i, k, j) triplets of mask_{P_C}(A.B) and the useful flops
 * sum 2 n_i n_k n_j (padding never counted).  Builds the task list if needed. */
cq_status cq_bsmm_work(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                       const cq_pattern *pC, int64_t *triplets_host, double *flops_host);

/* Tr(A.B) = sum_{(i,j) in P_A} sum_{a,b} A_ij[a,b] B_ji[b,a] (absent B blocks count zero);
 * deterministic FP64 two-level reduction.  Synchronises. */
cq_status cq_trace_prod(cq_ctx *ctx, const cq_pattern *pA, const double *A,
                        const cq_pattern *pB, const double *B, double *out_host);

/*
 * Tr(A.B) as cq_trace_prod computes it, for callers that cannot allocate device memory when
 * they need it: code whose device memory is owned by a framework with a fixed budget that
 * forbids raw cudaMalloc, latency-critical loops that must not pay for cudaMalloc (it can
 * synchronise the device), or callers that hold no context (a pattern outlives the context
 * that built it).  (The paper has no counterpart: this is an interface variant, not part of
 * the method.)
 *
 * It allocates nothing: its scratch, one FP64 partial per atom row, is a file-scope
 * __device__ array of 65536 doubles (512 KiB) that every GPU loading the library keeps until
 * the process exits; no cudaMalloc, cudaFree or allocating library routine is called.
 * pA, A, pB, B are as for cq_trace_prod (existing patterns and values); the work runs on
 * the device the patterns were built on (both must be on the same one, else
 * CQ_ERR_PATTERN).  out_dev is a device pointer that receives the trace; cuda_stream is
 * the stream to enqueue on (NULL: legacy default stream).  The call is asynchronous: read
 * out_dev after synchronising the stream.  Patterns of more than 65536 atoms are rejected
 * with CQ_ERR_INVALID.  On error, *message_host (if message_host is not NULL) points to a
 * static description.
 *
 * The first call on a device looks up the array's device address with that device current
 * (cudaGetSymbolAddress, a synchronising runtime call); later calls reuse it.  Every call
 * shares the one array and leaves its contents behind; each call overwrites the rows it
 * reads, but calls that overlap on the GPU (different streams or host threads) race on the
 * array and must be serialised by the caller.
 */
cq_status cq_trace_prod_static(const cq_pattern *pA, const double *A, const cq_pattern *pB,
                               const double *B, double *out_dev, void *cuda_stream,
                               const char **message_host);

/* Frobenius inner product <A, B> over the blocks of p.  Synchronises. */
cq_status cq_dot(cq_ctx *ctx, const cq_pattern *p, const double *A, const double *B,
                 double *out_host);

/* ---------------------------------------------------------------- overlap inversion */

/* T_0 = I / sigma on P_T, sigma = max_a sum_b |S_ab| (largest absolute scalar row sum of S,
 * which bounds its spectrum, so the Hotelling iteration converges).  Synchronises. */
cq_status cq_hotelling_init(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                            const cq_pattern *pT, double *T);

/*
 * One Hotelling step for T ~ S^-1 (Development Priorities: linear-scaling inversion of the
 * overlap): V = S.T on P_{rS+rT} (the whole product), resid = ||V - I||_F for the incoming
 * T, then T <- 2T - mask_{P_T}(T.V).  T is updated in place.  Synchronises.
 */
cq_status cq_hotelling_step(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                            const cq_pattern *pT, double *T, double *resid_host);

/*
 * Least-squares overlap inverse (Development Priorities: other ways to invert the overlap in
 * linear-scaling time): the T on P_T that minimises ||I - S T||_F,
 * found by linear conjugate gradients on the symmetric values of T, started from the T
 * passed in (e.g. cq_hotelling_init, or a Hotelling result to refine).  R = I - S T is kept
 * on P_{rS+rT}; the gradient on P_T is G = -(W + W^T) with W = mask_{P_T}(S R); each step
 * takes the exact minimiser along D (two products per step: S.D and S.R), then
 * D <- -G + (|G|^2 / |G_prev|^2) D.  Unlike Hotelling's truncated fixed point, the result
 * is the best inverse the pattern can hold.
 *   T          in: symmetric start on P_T; out: the last iterate (updated in place).
 *   max_iter   step limit (>= 0); gtol: stop once ||G||_F <= gtol ||G_0||_F (>= 0).
 *   resid_host, gnorm_host  NULL or host arrays of max_iter + 1 doubles: ||I - S T_k||_F and
 *              ||G_k||_F for the start (k = 0) and every iterate.
 *   iters_host NULL or the number of steps taken (history entries 0..*iters_host hold
 *              values).  After an error it is the last step whose entries were written (-1:
 *              none), so the caller knows which entries are valid.
 * Single cells only (batch patterns give CQ_ERR_INVALID); FP64; scratch owned by the
 * context.  A non-finite residual gives CQ_ERR_NUMERIC.  After an error T holds an
 * iterate of the run (possibly a partly applied step), not the start.  Synchronises every
 * step.
 */
cq_status cq_overlap_inverse_cg(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                                const cq_pattern *pT, double *T, int32_t max_iter,
                                double gtol, double *resid_host, double *gnorm_host,
                                int32_t *iters_host);

/* ---------------------------------------------------------------- density matrix */

/*
 * Palser-Manolopoulos start for the density-matrix optimisation (non-orthogonal form):
 * L = mask_L[(lambda/N)(mu T - T H T) + (n_occ/N) T], N = number of orbitals,
 * mu = Tr(TH)/N, lambda = min(n_occ/(h_max - mu), (N - n_occ)/(mu - h_min)) with h_min,
 * h_max the Gershgorin bounds of TH.  T ~ S^-1 on P_T; H on P_S.  Synchronises.
 */
cq_status cq_pm_guess(cq_ctx *ctx, const cq_pattern *pS, const double *S, const double *H,
                      const cq_pattern *pT, const double *T, const cq_pattern *pL,
                      double *L, double n_occ);

/* The same for a batch: n_occ_host[c] occupied states in cell c, and mu, lambda, the
 * Gershgorin bounds and N per cell.  cq_pm_guess is this call on a one-cell pattern. */
cq_status cq_pm_guess_cells(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                            const double *H, const cq_pattern *pT, const double *T,
                            const cq_pattern *pL, double *L, const double *n_occ_host);

/* One McWeeny purification step L <- mask_L(3LSL - 2LSLSL), every intermediate kept on its
 * full range (r_L + r_S, 2 r_S + r_L, 2 r_L) so the masked result is exact. */
cq_status cq_mcweeny_step(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                          const cq_pattern *pL, double *L);

/* Per-step record of an LNV step. */
typedef struct {
    double energy;      /* E = 2 Tr(K H), hartree                                   */
    double n_elec;      /* N = 2 Tr(K S)                                            */
    double mu;          /* chemical potential <G_E,G_N>/<G_N,G_N> at the new L       */
    double gnorm;       /* RMS of G = G_E - mu G_N over the values of P_L            */
    double alpha;       /* accepted step length                                     */
    int32_t restart;    /* 1 if the search direction was reset to -G                */
    int32_t fallback;   /* 1 if the cubic had no positive minimum (alpha = 2 alpha2) */
    int32_t n_corr;     /* electron-number corrections applied after the step        */
    int32_t n_products; /* block products the step ran                              */
    double flops;       /* useful flops of those products (sum 2 n_i n_k n_j)         */
} cq_lnv_report;

/*
 * Li-Nunes-Vanderbilt minimisation (Development Priorities: linear-scaling optimisation of
 * the density matrix) of E = 2 Tr(K H) at N = 2 Tr(K S) = n_electrons, K = 3LSL - 2LSLSL,
 * over L on P_L.  S and H share pattern pS; L (in/out, on pL) is the start (e.g. from
 * cq_pm_guess) and always holds the current iterate.  Create evaluates E, N and the
 * gradients and applies electron-number corrections; each step then does a Polak-Ribiere
 * direction projected orthogonal to G_N, an exact cubic line search of E - mu N from two
 * trial points, the update and at most five corrections while |N - N_e| > 1e-10 N_e.
 * The object keeps pointers to S, H and L: they must outlive it.  Synchronises.
 */
cq_status cq_lnv_create(cq_ctx *ctx, const cq_pattern *pS, const double *S, const double *H,
                        const cq_pattern *pL, double *L, double n_electrons,
                        cq_precision prec, cq_lnv **out);
/* Batch version: n_electrons_host[c] electrons in cell c; every scalar of the minimisation
 * (mu, CG coefficients, line search, corrections) is per cell, the products are shared
 * launches.  cq_lnv_create is this call on a one-cell pattern. */
cq_status cq_lnv_create_cells(cq_ctx *ctx, const cq_pattern *pS, const double *S,
                              const double *H, const cq_pattern *pL, double *L,
                              const double *n_electrons_host, cq_precision prec,
                              cq_lnv **out);
/* One step; report_host receives one cq_lnv_report per cell (one for a single cell). */
cq_status cq_lnv_step(cq_lnv *lnv, cq_lnv_report *report_host);
/* Number of cells of the LNV object. */
int32_t cq_lnv_cells(const cq_lnv *lnv);
/* Switch the precision of the products of later steps (e.g. split-BF16 steps followed by
 * FP64 refinement sweeps).  The current L, E, N and gradients are re-evaluated in the new
 * precision (with electron-number corrections) so the next step starts from consistent
 * values; the search history is reset.  Synchronises. */
cq_status cq_lnv_set_precision(cq_lnv *lnv, cq_precision prec);
/* Precondition the search directions of later steps (Development Priorities: the overlap
 * inversion feeding the density-matrix optimisation; T applied on both sides of the
 * covariant gradient gives the contravariant direction).  pT, T: an approximate S^-1 on
 * its own range-cutoff pattern (e.g. from cq_hotelling), device values in pT's layout; same
 * atoms and basis as the LNV patterns.  Each step then forms Z = sym(mask_L(T G T)) with
 * two more products (T G on the pattern of range r_T + r_L, owned by the context) and uses
 * Z where the plain step uses G: D = -Z + beta D_prev with
 * beta = max(0, <G, Z - Z_prev> / <G_prev, Z_prev>), restarts to -Z, and the first trial
 * step 0.1 sqrt(n) / ||Z||.  With T = identity the steps are those of the plain gradient.
 * T is copied (the caller keeps its buffer); pT must outlive the preconditioner.  T = NULL
 * or pT = NULL switches it off, and so does a failed call.  The search history is reset
 * either way.  Single cells only: a batched LNV object (cq_lnv_create_cells) gives
 * CQ_ERR_INVALID.  Synchronises. */
cq_status cq_lnv_set_preconditioner(cq_lnv *lnv, const cq_pattern *pT, const double *T);
/* Current E, N, mu and RMS gradient (as after the last evaluation), one report per cell. */
cq_status cq_lnv_state(const cq_lnv *lnv, cq_lnv_report *report_host);
/* Useful flops of one LNV step's products (full evaluation + two trial points, plus the two
 * preconditioner products when one is set). */
cq_status cq_lnv_step_flops(cq_lnv *lnv, double *flops_host);
void cq_lnv_destroy(cq_lnv *lnv);

/* ---------------------------------------------------------------- learned initial guess */

/*
 * A small network that predicts the density-matrix blocks of L from each atom pair's local
 * environment, as a start for the LNV minimisation (which refines it and falls back to
 * cq_pm_guess when its start is poor).  The paper's density-matrix optimisation needs a
 * start; a learned one is this library's addition.  Pairs are the blocks (i, j), i <= j, of
 * a one-cell P_L with a uniform basis of 4 or 9 orbitals; (j, i) is the transpose.
 *
 * Pair frame: e3 along r_j - r_i (on-site: toward i's nearest neighbour); e1 toward the atom
 * nearest the midpoint (other than i, j; ties to the lowest index; atoms on the axis
 * skipped), orthogonalised; e2 = e3 x e1.  Descriptor (64 floats): 10 Gaussians of r_ij
 * (centres 1.6p, width 1.6) and, over atoms k of row i within 8 bohr of the midpoint,
 * sum_k h_n(|r_k - m|) Y_a(frame direction) for 6 radial Gaussians (centres 1.6n, width
 * 1.2, cosine cut at 8) and 9 real harmonics (1, z, x, y, (3z^2-1)/2, xz, yz, (x^2-y^2)/2,
 * xy).  Targets: the block in the pair frame, D L_ij D^T (D the s/p/d orbital rotation),
 * 81 floats (zero-padded for 4 orbitals).  Network: 64 -> 256 -> 256 -> 256 -> 81, SiLU
 * hidden activations, BF16 weights (FP32 master copy) and FP32 accumulation, inputs and
 * outputs normalised per column.  Training: MSE on normalised targets, Adam (0.9, 0.999,
 * 1e-8).  fp32_weights != 0 makes the forward pass read the FP32 weights (test mode).
 */
typedef struct cq_guess cq_guess;
cq_status cq_guess_create(cq_ctx *ctx, uint64_t seed, int32_t fp32_weights, cq_guess **out);
void cq_guess_destroy(cq_guess *g);
/* Number of pair blocks (i <= j) of pL. */
cq_status cq_guess_pairs(cq_ctx *ctx, const cq_pattern *pL, int64_t *n_pairs_host);
/* Descriptors (n_pairs x 64), frames (n_pairs x 9: rows e1, e2, e3) and, if pairs_dev is
 * not NULL, the block index of each pair (n_pairs int32). */
cq_status cq_guess_descriptors(cq_ctx *ctx, const cq_pattern *pL, float *desc_dev,
                               float *frames_dev, int32_t *pairs_dev);
/* Pair-frame targets (n_pairs x 81) of a converged L on pL. */
cq_status cq_guess_targets(cq_ctx *ctx, const cq_pattern *pL, const double *L,
                           const float *frames_dev, float *targets_dev);
/* Per-column normalisation of inputs and targets from training data (rows samples). */
cq_status cq_guess_fit_scale(cq_guess *g, const float *desc_dev, const float *targets_dev,
                             int64_t rows);
cq_status cq_guess_set_scale(cq_guess *g, const float *in_mean_host, const float *in_scale_host,
                             const float *out_mean_host, const float *out_scale_host);
/* Copy the FP32 weights and biases (layer by layer, row-major in x out) to (set = 0) or from
 * (set != 0) host arrays of n_w and n_b floats; either pointer may be NULL. */
cq_status cq_guess_params(cq_guess *g, float *w_host, float *b_host, int64_t *n_w,
                          int64_t *n_b, int32_t set);
/* One Adam step on a minibatch of rows samples (raw targets; lr = 0: loss and gradients
 * only).  Optional host outputs: mean-square loss of the normalised targets, gradients; the
 * call synchronises only when it fills one of them (else it is asynchronous on the context
 * stream).  Every step also adds its squared-error sum and its row count to the device-side
 * running sums that cq_guess_loss_sum reads. */
cq_status cq_guess_train_step(cq_guess *g, const float *desc_dev, const float *targets_dev,
                              int64_t rows, float lr, float *loss_host, float *grad_w_host,
                              float *grad_b_host);
/* The running sums of the training steps since the last reset: *sq_sum_host = sum of the
 * squared errors of the normalised targets (81 per row), *rows_host = rows; synchronises.
 * reset != 0 sets both to zero after reading.  The mean-square loss over those steps is
 * sq_sum / (81 rows). */
cq_status cq_guess_loss_sum(cq_guess *g, double *sq_sum_host, int64_t *rows_host, int32_t reset);
/* Normalised network outputs (rows x 81). */
cq_status cq_guess_forward(cq_guess *g, const float *desc_dev, int64_t rows, float *out_dev);
/* L on pL from the network: every block predicted, rotated back, (j, i) = (i, j)^T. */
cq_status cq_guess_apply(cq_guess *g, const cq_pattern *pL, double *L);

#ifdef __cplusplus
}
#endif

#endif /* CQ_H */
