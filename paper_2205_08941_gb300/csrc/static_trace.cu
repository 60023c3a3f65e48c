// Tr(A.B) without any device allocation.
//
// cq_trace_prod reduces through scratch that the context allocates on first use.  Some
// callers cannot allocate device memory at the time they need a trace: code whose device
// memory is owned by a host framework with a fixed budget that forbids raw cudaMalloc,
// latency-critical loops that must not pay for cudaMalloc (which can synchronise the
// device), or callers that hold no context at all (patterns outlive the context that
// built them).  cq_trace_prod_static serves them: its scratch -- one partial sum per atom
// row -- lives in a file-scope __device__ array of CQ_STATIC_TRACE_MAX_ROWS doubles
// (512 KiB) that every GPU which loads the library keeps until the process exits.  It calls
// no cudaMalloc, cudaFree or allocating library routine.
//
// The caller passes patterns and values that already exist (patterns from cq_pattern_build
// hold their index arrays on the device they were built on, which the pattern records) and
// a device pointer for the result.  Every call shares the one array, which keeps the last
// call's contents; each call overwrites the rows it uses before reading them, so nothing
// needs clearing, but calls that overlap on the GPU (on different streams, or from several
// host threads) race on the array and must be serialised by the caller.
#include <cstring>
#include <mutex>

#include "cq_internal.cuh"

#define CQ_STATIC_TRACE_MAX_ROWS 65536
#define CQ_STATIC_TRACE_MAX_DEVICES 64

static __device__ __align__(256) double g_trace_rows[CQ_STATIC_TRACE_MAX_ROWS];

namespace {

// one warp per atom row i: sum over blocks (i, j) of P_A of <A_ij, (B_ji)^T>, B_ji found by
// binary search in row j of P_B (absent blocks count zero)
__global__ void k_trace_rows(int n_atoms, const int64_t *a_rp, const int32_t *a_col,
                             const int32_t *nb, const int64_t *a_off, const int64_t *b_rp,
                             const int32_t *b_col, const int64_t *b_off, const double *A,
                             const double *B, double *rows)
{
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n_atoms) return;
    double s = 0.0;
    const int ni = nb[i];
    for (int64_t e = a_rp[i]; e < a_rp[i + 1]; ++e) {
        const int j = a_col[e];
        int64_t lo = b_rp[j], hi = b_rp[j + 1];
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (b_col[mid] < i)
                lo = mid + 1;
            else
                hi = mid;
        }
        if (lo >= b_rp[j + 1] || b_col[lo] != i) continue;
        const int nj = nb[j];
        const double *a = A + a_off[e];
        const double *b = B + b_off[lo];
        for (int q = lane; q < ni * nj; q += 32) {
            const int r = q / nj, c = q - r * nj;
            s = fma(a[q], b[c * ni + r], s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) rows[i] = s;
}

// one CTA folds the row partials in a fixed order
__global__ void k_trace_rows_sum(int n, const double *rows, double *out)
{
    __shared__ double sh[256];
    double s = 0.0;
    for (int e = threadIdx.x; e < n; e += 256) s += rows[e];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

std::mutex g_setup_mutex;
double *g_rows_addr[CQ_STATIC_TRACE_MAX_DEVICES] = {nullptr};

}  // namespace

extern "C" cq_status cq_trace_prod_static(const cq_pattern *pA, const double *A,
                                          const cq_pattern *pB, const double *B, double *out_dev,
                                          void *cuda_stream, const char **message_host)
{
    auto fail = [&](cq_status st, const char *msg) {
        if (message_host) *message_host = msg;
        return st;
    };
    if (message_host) *message_host = "";
    if (!pA || !pB || !out_dev || (!A && pA->n_values) || (!B && pB->n_values))
        return fail(CQ_ERR_INVALID, "trace_prod_static: null argument");
    if (!cq_same_atoms(pA, pB))
        return fail(CQ_ERR_PATTERN, "trace_prod_static: patterns over different atoms");
    const int n = pA->geo->n_atoms;
    if (n > CQ_STATIC_TRACE_MAX_ROWS)
        return fail(CQ_ERR_INVALID,
                    "trace_prod_static: more than 65536 atoms (the static scratch holds one "
                    "partial per atom row); use cq_trace_prod");
    // the device the patterns were built on (recorded in their geometry, so it survives
    // the destruction of the context that built them)
    const int device = pA->geo->device;
    if (pB->geo->device != device)
        return fail(CQ_ERR_PATTERN, "trace_prod_static: patterns on different devices");
    if (device < 0 || device >= CQ_STATIC_TRACE_MAX_DEVICES)
        return fail(CQ_ERR_INVALID, "trace_prod_static: device ordinal beyond 63");
    int current = 0;
    if (cudaGetDevice(&current) != cudaSuccess) {
        cudaGetLastError();
        return fail(CQ_ERR_CUDA, "trace_prod_static: cudaGetDevice failed");
    }
    if (current != device && cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return fail(CQ_ERR_CUDA, "trace_prod_static: cudaSetDevice failed");
    }
    double *rows = nullptr;
    {
        // set-up once per device, with that device current: the array's device address
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_rows_addr[device]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_trace_rows);
            if (e != cudaSuccess) {
                cudaGetLastError();
                if (current != device) cudaSetDevice(current);
                return fail(CQ_ERR_CUDA, "trace_prod_static: cudaGetSymbolAddress failed");
            }
            g_rows_addr[device] = (double *)p;
        }
        rows = g_rows_addr[device];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (n > 0) {
        k_trace_rows<<<(n + 7) / 8, 256, 0, s>>>(
            n, pA->row_ptr.as<int64_t>(), pA->col.as<int32_t>(), pA->geo->nb.as<int32_t>(),
            pA->val_off.as<int64_t>(), pB->row_ptr.as<int64_t>(), pB->col.as<int32_t>(),
            pB->val_off.as<int64_t>(), A, B, rows);
    }
    k_trace_rows_sum<<<1, 256, 0, s>>>(n, rows, out_dev);
    cq_count_launch(n > 0 ? 2 : 1);
    const cudaError_t e = cudaGetLastError();
    if (current != device) cudaSetDevice(current);
    if (e != cudaSuccess) return fail(CQ_ERR_CUDA, "trace_prod_static: kernel launch failed");
    return CQ_OK;
}
