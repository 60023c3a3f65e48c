// Internal structures of libcq: context, geometry, pattern, task lists, scratch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/cq.h"

#define CQ_MAX_NB 16          // largest orbital count per atom on the device path
#define CQ_ROW_CAP 8192       // largest number of blocks in one pattern row
#define CQ_RED_SLOTS 8192     // device scalar slots (8 per cell for up to 1024 cells)
#define CQ_MAX_CELLS 1024

struct cq_ctx;

// Device buffer owned by a context; counts against the context's memory cap.
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    cq_ctx *ctx = nullptr;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf();
    template <class T> T *as() const { return static_cast<T *>(ptr); }
};

// Atom positions, box and basis shared by every pattern built on the same geometry.
struct Geometry {
    uint64_t id = 0;
    int device = 0;                 // CUDA device holding the pattern arrays (kept after the
                                    // context is destroyed)
    int32_t n_atoms = 0;
    double box[3] = {0, 0, 0};
    std::vector<double> pos_host;   // n_atoms * 3
    std::vector<int32_t> nb_host;   // n_atoms
    int64_t n_orb = 0;
    int uniform_nb = 0;             // orbital count if every atom has the same, else 0
    DevBuf pos, nb;                 // device copies
    // batches: n_cells independent periodic cells, atoms of cell c = [cell_start[c],
    // cell_start[c+1]), each with its own box (boxes[3c..3c+2]); one cell otherwise
    int n_cells = 1;
    std::vector<int32_t> cell_start;  // n_cells + 1
    std::vector<double> boxes;        // 3 * n_cells
    std::vector<int64_t> cell_orb;    // orbitals per cell
    DevBuf cell_of, boxes_dev, cell_start_dev;
};

// (i, k, j) task list of mask_{P_C}(A.B), sorted by C block then k ascending.
struct TaskList {
    int64_t n_c = 0;
    int64_t n_tasks = 0;
    double flops = 0.0;
    DevBuf seg;     // int64 [n_c + 1]
    DevBuf tasks;   // int2  [n_tasks]: (A block, B block), filled on first FP64 use
    bool filled = false;
    DevBuf c_rowitem;  // int64 [n_c + 1] prefix of n_i over C blocks (bases other than 4, 9)
    int64_t n_items = 0;  // scalar C rows (sum of n_i over C blocks)
    mutable int q = 0;    // lanes per C row of the FP64 kernel chosen by the autotuner (0: none)
};

struct cq_pattern {
    cq_ctx *ctx = nullptr;
    uint64_t id = 0;
    std::shared_ptr<Geometry> geo;
    double range = 0.0;
    int64_t n_blocks = 0;
    int64_t n_values = 0;
    int64_t n_scalars = 0;           // sum of nb[i]*nb[j] over blocks (no padding)
    int64_t max_row = 0;
    int uniform = 0;                 // padded block stride if the basis is uniform, else 0
    DevBuf row_ptr;                  // int64 [n+1]
    DevBuf col;                      // int32 [n_blocks]
    DevBuf row;                      // int32 [n_blocks]
    DevBuf val_off;                  // int64 [n_blocks]
    DevBuf transpose;                // int64 [n_blocks]
    std::vector<int64_t> row_ptr_host;
    bool owned_by_ctx = false;
    // per-cell range and the block / value segments of each cell (contiguous, since the
    // cells' atoms are)
    std::vector<double> ranges;
    std::vector<int64_t> seg_blk, seg_val, seg_scalars;  // n_cells + 1 / n_cells
    DevBuf seg_blk_dev, seg_val_dev;
    int n_cells() const { return (int)ranges.size(); }
};

struct cq_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    int64_t mem_limit = 0;
    int64_t mem_used = 0;
    uint64_t next_id = 1;
    int num_sms = 0;
    DevBuf flag;                     // int32 device error word
    DevBuf red;                      // reduction partials
    DevBuf red_out;                  // reduction results (pinned-copy source)
    double *host_out = nullptr;      // pinned host scalars
    std::map<std::tuple<uint64_t, uint64_t, uint64_t>, std::unique_ptr<TaskList>> tasks;
    std::map<std::tuple<uint64_t, uint64_t, int>, std::unique_ptr<DevBuf>> maps;
    std::map<std::pair<uint64_t, std::vector<double>>, cq_pattern *> derived;
    std::map<std::string, std::unique_ptr<DevBuf>> scratch;
    std::vector<cq_pattern *> live_patterns;
    std::vector<cq_lnv *> live_lnv;
    // other cached per-pattern data, keyed (kind, id, id, id); entries naming a destroyed
    // pattern's id are dropped with it
    std::map<std::tuple<int, uint64_t, uint64_t, uint64_t>, std::shared_ptr<void>> aux;
    // product-kernel timing
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    size_t ev_used = 0;
    double timed_flops = 0.0;
    double timed_mma_flops = 0.0;
    bool autotune = false;           // time the FP64 lane splits on a product's first use
    bool graphs = false;             // replay LNV evaluation phases as CUDA graphs
    bool capturing = false;          // a graph capture is open on the stream
    uint64_t scratch_gen = 0;        // bumped whenever a scratch buffer is reallocated
    int64_t test_wait_cycles = 0;    // > 0: split kernels make their first wait run out
};

// Record a timing event pair around a product launch when timing is on.
void cq_timing_begin(cq_ctx *ctx, double flops, double mma_flops = 0.0);
void cq_timing_end(cq_ctx *ctx);

// ---------------------------------------------------------------- helpers (ctx.cu)
cq_status cq_fail(cq_ctx *ctx, cq_status st, const std::string &msg);
cq_status cq_check_cuda(cq_ctx *ctx, cudaError_t e, const char *what);
cq_status cq_alloc(cq_ctx *ctx, DevBuf &buf, size_t bytes);
// Scratch buffer by name, grown (never shrunk) to at least `bytes`.
cq_status cq_scratch(cq_ctx *ctx, const std::string &name, size_t bytes, void **out);
// Exclusive scan of int64 counts (n entries) into out (n + 1 entries), out[n] = total.
cq_status cq_scan_i64(cq_ctx *ctx, const int64_t *in, int64_t *out, int64_t n);
// Read and clear the device error word (synchronises).
cq_status cq_read_flag(cq_ctx *ctx, int32_t *flag);

// ---------------------------------------------------------------- patterns (pattern.cu)
cq_status cq_pattern_build_geo(cq_ctx *ctx, std::shared_ptr<Geometry> geo,
                               const std::vector<double> &ranges, cq_pattern **out);
// Pattern of the same geometry with per-cell range ca*range_a[c] + cb*range_b[c], owned and
// cached by the context.
cq_status cq_pattern_derived(cq_ctx *ctx, const cq_pattern *base, double ca,
                             const cq_pattern *pa, double cb, const cq_pattern *pb,
                             cq_pattern **out);
bool cq_same_atoms(const cq_pattern *a, const cq_pattern *b);

// ---------------------------------------------------------------- tasks (tasks.cu)
cq_status cq_get_tasks(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                       const cq_pattern *pC, TaskList **out);
// Fill the (A block, B block) pairs of a counted task list (first FP64 product on it).
cq_status cq_fill_tasks(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                        const cq_pattern *pC, TaskList *tl);
// Map from the blocks of pDst to the blocks of pSrc holding (i, j) (or (j, i) when
// transpose), -1 when absent.  Cached in the context.
cq_status cq_get_map(cq_ctx *ctx, const cq_pattern *pSrc, const cq_pattern *pDst,
                     int transpose, const int64_t **out);

// ---------------------------------------------------------------- products
cq_status cq_bsmm_f64(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                      const double *A, const cq_pattern *pB, const double *B, double beta,
                      const cq_pattern *pC, double *C);
// Lane split the FP64 kernel uses for a task list (tuned if the autotuner ran, else the
// mean-segment heuristic).
int cq_lane_split(const TaskList *tl);
cq_status cq_bsmm_split(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                        const double *A, const cq_pattern *pB, const double *B, double beta,
                        const cq_pattern *pC, double *C);
cq_status cq_bsmm_emu(cq_ctx *ctx, const TaskList *tl, double alpha, const cq_pattern *pA,
                      const double *A, const cq_pattern *pB, const double *B, double beta,
                      const cq_pattern *pC, double *C);

// ---------------------------------------------------------------- reductions (reduce.cu)
// All scalar results land in ctx->red_out[slot] on the device; cq_fetch copies them out.
cq_status cq_trace_dev(cq_ctx *ctx, const cq_pattern *pA, const double *A,
                       const cq_pattern *pB, const double *B, int slot);
cq_status cq_dot_dev(cq_ctx *ctx, const cq_pattern *p, const double *A, const double *B,
                     int slot);
cq_status cq_frob2_minus_identity_dev(cq_ctx *ctx, const cq_pattern *p, const double *M,
                                      int slot);
// slots: [slot] = min(centre - radius), [slot+1] = max(centre + radius), [slot+2] = max |row|
cq_status cq_row_bounds_dev(cq_ctx *ctx, const cq_pattern *p, const double *M, int slot);
cq_status cq_fetch(cq_ctx *ctx, int first, int count, double *host);

// ---------------------------------------------------------------- elementwise (reduce.cu)
// y <- a*x + b*y over n doubles (b == 0: y not read)
cq_status cq_axpby(cq_ctx *ctx, int64_t n, double a, const double *x, double b, double *y);
// dst <- s * (src_ij or src_ji^T) + b * dst on pDst; absent source blocks read as zero
cq_status cq_gather(cq_ctx *ctx, const cq_pattern *pSrc, const double *src,
                    const cq_pattern *pDst, double *dst, int transpose, double s, double b);
// M <- s * I on the diagonal blocks of p, zero elsewhere
cq_status cq_set_identity(cq_ctx *ctx, const cq_pattern *p, double *M, double s);
// G_E = 2[3(Z + Z^T) - 2(R1 + R1^T + R2)], G_N = 12(U - R3) on P_L
cq_status cq_lnv_gradients(cq_ctx *ctx, const cq_pattern *pL, const cq_pattern *pU,
                           const double *Z, const double *U, const double *R1,
                           const double *R2, const double *R3, double *GE, double *GN);

// ---------------------------------------------------------------- per-cell (batches)
// One result per cell into red_out[slot + c] (n_cells > 1; contiguous segments).
cq_status cq_trace_seg_dev(cq_ctx *ctx, const cq_pattern *pA, const double *A,
                           const cq_pattern *pB, const double *B, int slot);
cq_status cq_dot_seg_dev(cq_ctx *ctx, const cq_pattern *p, const double *A, const double *B,
                         int slot);
// per cell: [slot + 3c] = min(centre - radius), [+1] = max(centre + radius), [+2] = max |row|
cq_status cq_row_bounds_seg_dev(cq_ctx *ctx, const cq_pattern *p, const double *M, int slot);
// y <- a[c]*x + b[c]*y on each cell's values (coefficients copied from the host)
cq_status cq_axpby_seg(cq_ctx *ctx, const cq_pattern *p, const double *a, const double *x,
                       const double *b, double *y);
// M <- s[c] * I on each cell's diagonal blocks, zero elsewhere
cq_status cq_set_identity_seg(cq_ctx *ctx, const cq_pattern *p, double *M, const double *s);

// Launch-count bookkeeping (kernels this library launched; read by the bench).
void cq_count_launch(int64_t n = 1);
// While a graph is captured on this thread, launches are counted into the graph (and
// added to the total each time it is replayed).
void cq_capture_counting(bool on);
int64_t cq_capture_launches(void);

static inline int64_t cq_pad2(int64_t x) { return (x + 1) & ~int64_t(1); }

// Called by cq_ctx_destroy for LNV objects still alive: they stop touching the context.
void cq_lnv_detach(cq_lnv *s);
// G_N = 12(U - R3) only (the electron-number gradient) on P_L.
cq_status cq_lnv_gradient_n(cq_ctx *ctx, const cq_pattern *pL, const cq_pattern *pU,
                            const double *U, const double *R3, double *GN);
// G_E = 2[3(Z + Z^T) - 2((R1 + R1^T) + R2)] only, on P_L.
cq_status cq_lnv_gradient_e(cq_ctx *ctx, const cq_pattern *pL, const cq_pattern *pU,
                            const double *Z, const double *R1, const double *R2, double *GE);
