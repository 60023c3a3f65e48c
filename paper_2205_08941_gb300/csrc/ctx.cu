// Context, errors, device memory, the int64 scan utility and the public entry points that
// are thin wrappers (patterns, products, traces).
#include <atomic>
#include <cmath>
#include <cstring>

#include "cq_internal.cuh"

static std::atomic<int64_t> g_launches{0};
extern "C" int64_t cq_kernel_launches(void) { return g_launches.load(); }
static thread_local bool t_capturing = false;
static thread_local int64_t t_captured = 0;
void cq_count_launch(int64_t n)
{
    if (t_capturing)
        t_captured += n;
    else
        g_launches.fetch_add(n);
}
void cq_capture_counting(bool on)
{
    t_capturing = on;
    if (on) t_captured = 0;
}
int64_t cq_capture_launches(void) { return t_captured; }

DevBuf::~DevBuf()
{
    if (ptr) {
        cudaFree(ptr);
        if (ctx) ctx->mem_used -= (int64_t)bytes;
    }
}

cq_status cq_fail(cq_ctx *ctx, cq_status st, const std::string &msg)
{
    if (ctx) ctx->err = msg;
    return st;
}

cq_status cq_check_cuda(cq_ctx *ctx, cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return CQ_OK;
    cudaGetLastError();
    return cq_fail(ctx, e == cudaErrorMemoryAllocation ? CQ_ERR_NOMEM : CQ_ERR_CUDA,
                   std::string(what) + ": " + cudaGetErrorString(e));
}

cq_status cq_alloc(cq_ctx *ctx, DevBuf &buf, size_t bytes)
{
    if (buf.ptr) {
        cudaFree(buf.ptr);
        if (buf.ctx) buf.ctx->mem_used -= (int64_t)buf.bytes;
        buf.ptr = nullptr;
        buf.bytes = 0;
    }
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    if (ctx->mem_limit > 0 && ctx->mem_used + (int64_t)bytes > ctx->mem_limit)
        return cq_fail(ctx, CQ_ERR_NOMEM, "context memory limit reached");
    cudaError_t e = cudaMalloc(&buf.ptr, bytes);
    if (e != cudaSuccess) {
        buf.ptr = nullptr;
        return cq_check_cuda(ctx, e, "cudaMalloc");
    }
    buf.bytes = bytes;
    buf.ctx = ctx;
    ctx->mem_used += (int64_t)bytes;
    return CQ_OK;
}

cq_status cq_scratch(cq_ctx *ctx, const std::string &name, size_t bytes, void **out)
{
    auto &slot = ctx->scratch[name];
    if (!slot) slot.reset(new DevBuf());
    if (slot->bytes < bytes) {
        if (ctx->capturing)
            return cq_fail(ctx, CQ_ERR_INVALID, "scratch growth inside a graph capture");
        // make sure no queued kernel still uses the old buffer
        cq_status st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
        if (st != CQ_OK) return st;
        st = cq_alloc(ctx, *slot, bytes);
        if (st != CQ_OK) return st;
        ctx->scratch_gen++;
    }
    *out = slot->ptr;
    return CQ_OK;
}

// ---------------------------------------------------------------- int64 exclusive scan

namespace {
constexpr int SCAN_T = 512;
constexpr int SCAN_I = 8;
constexpr int64_t SCAN_TILE = SCAN_T * SCAN_I;

__device__ int64_t block_exclusive(int64_t v, int64_t *total)
{
    __shared__ int64_t ws[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t s = lane < SCAN_T / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCAN_T / 32) ws[lane] = s;
    }
    __syncthreads();
    const int64_t off = wid ? ws[wid - 1] : 0;
    *total = ws[SCAN_T / 32 - 1];
    __syncthreads();
    return off + x - v;
}

__global__ void k_tile_sums(const int64_t *in, int64_t n, int64_t *sums)
{
    const int64_t base = blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t s = 0;
    for (int e = 0; e < SCAN_I; ++e)
        if (base + e < n) s += in[base + e];
    int64_t tot;
    block_exclusive(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_tile_scan(const int64_t *in, int64_t n, const int64_t *tile_off,
                            int64_t *out)
{
    const int64_t base = blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_I;
    int64_t v[SCAN_I];
    int64_t s = 0;
    for (int e = 0; e < SCAN_I; ++e) {
        v[e] = (base + e < n) ? in[base + e] : 0;
        s += v[e];
    }
    int64_t tot;
    int64_t run = block_exclusive(s, &tot) + (tile_off ? tile_off[blockIdx.x] : 0);
    for (int e = 0; e < SCAN_I; ++e) {
        if (base + e < n) out[base + e] = run;
        run += v[e];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0)
        out[n] = (tile_off ? tile_off[blockIdx.x] : 0) + tot;
}

cq_status scan_level(cq_ctx *ctx, const int64_t *in, int64_t *out, int64_t n, int level)
{
    const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles <= 1) {
        k_tile_scan<<<1, SCAN_T, 0, ctx->stream>>>(in, n, nullptr, out);
        cq_count_launch();
        return cq_check_cuda(ctx, cudaGetLastError(), "scan");
    }
    void *p1, *p2;
    cq_status st = cq_scratch(ctx, "scan_sums" + std::to_string(level),
                              (size_t)tiles * sizeof(int64_t), &p1);
    if (st != CQ_OK) return st;
    st = cq_scratch(ctx, "scan_offs" + std::to_string(level),
                    (size_t)(tiles + 1) * sizeof(int64_t), &p2);
    if (st != CQ_OK) return st;
    k_tile_sums<<<(unsigned)tiles, SCAN_T, 0, ctx->stream>>>(in, n, (int64_t *)p1);
    cq_count_launch();
    st = scan_level(ctx, (int64_t *)p1, (int64_t *)p2, tiles, level + 1);
    if (st != CQ_OK) return st;
    k_tile_scan<<<(unsigned)tiles, SCAN_T, 0, ctx->stream>>>(in, n, (int64_t *)p2, out);
    cq_count_launch();
    return cq_check_cuda(ctx, cudaGetLastError(), "scan");
}
}  // namespace

cq_status cq_scan_i64(cq_ctx *ctx, const int64_t *in, int64_t *out, int64_t n)
{
    if (n == 0)
        return cq_check_cuda(ctx, cudaMemsetAsync(out, 0, sizeof(int64_t), ctx->stream),
                             "scan");
    return scan_level(ctx, in, out, n, 0);
}

// Device error bits that asynchronous kernels leave for the next synchronising call (the
// pattern and scatter bits are read by their own calls before they return).
constexpr int32_t CQ_FLAG_WAIT_TIMEOUT = 16;

cq_status cq_read_flag(cq_ctx *ctx, int32_t *flag)
{
    cq_status st = cq_check_cuda(
        ctx, cudaMemcpyAsync(ctx->host_out, ctx->flag.ptr, sizeof(int32_t),
                             cudaMemcpyDeviceToHost, ctx->stream), "flag read");
    if (st != CQ_OK) return st;
    st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    if (st != CQ_OK) return st;
    std::memcpy(flag, ctx->host_out, sizeof(int32_t));
    if (!*flag) return CQ_OK;
    st = cq_check_cuda(ctx, cudaMemsetAsync(ctx->flag.ptr, 0, 4, ctx->stream), "flag");
    if (st == CQ_OK && (*flag & CQ_FLAG_WAIT_TIMEOUT))
        return cq_fail(ctx, CQ_ERR_TIMEOUT,
                       "split product: a tensor-core wait ran out; the result is incomplete");
    return st;
}

// Copies the flag word into the last pinned slot with the stream's other work; after the
// stream is synchronised, reports (and clears) a wait that ran out on the device.
static cq_status queue_flag_read(cq_ctx *ctx)
{
    return cq_check_cuda(ctx, cudaMemcpyAsync(ctx->host_out + CQ_RED_SLOTS - 1, ctx->flag.ptr,
                                              sizeof(int32_t), cudaMemcpyDeviceToHost,
                                              ctx->stream), "flag read");
}

static cq_status check_async_flag(cq_ctx *ctx)
{
    int32_t f;
    std::memcpy(&f, ctx->host_out + CQ_RED_SLOTS - 1, sizeof(int32_t));
    if (!(f & CQ_FLAG_WAIT_TIMEOUT)) return CQ_OK;
    cudaMemsetAsync(ctx->flag.ptr, 0, 4, ctx->stream);
    return cq_fail(ctx, CQ_ERR_TIMEOUT,
                   "split product: a tensor-core wait ran out; the result is incomplete");
}

cq_status cq_fetch(cq_ctx *ctx, int first, int count, double *host)
{
    cq_status st = cq_check_cuda(
        ctx, cudaMemcpyAsync(ctx->host_out, ctx->red_out.as<double>() + first,
                             sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream),
        "scalar read");
    if (st != CQ_OK) return st;
    if ((st = queue_flag_read(ctx)) != CQ_OK) return st;
    st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    if (st != CQ_OK) return st;
    if ((st = check_async_flag(ctx)) != CQ_OK) return st;
    for (int e = 0; e < count; ++e) {
        host[e] = ctx->host_out[e];
        if (!std::isfinite(host[e]))
            return cq_fail(ctx, CQ_ERR_NUMERIC, "non-finite scalar result");
    }
    return CQ_OK;
}

// ---------------------------------------------------------------- public: context

extern "C" cq_status cq_ctx_create(int device, void *cuda_stream, cq_ctx **out)
{
    if (!out) return CQ_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CQ_ERR_CUDA;
    }
    if (cudaSetDevice(device) != cudaSuccess) return CQ_ERR_CUDA;
    cq_ctx *ctx = new cq_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cq_alloc(ctx, ctx->flag, 16) != CQ_OK ||
        cq_alloc(ctx, ctx->red_out, CQ_RED_SLOTS * 8) != CQ_OK ||
        cudaMallocHost(&ctx->host_out, CQ_RED_SLOTS * sizeof(double)) != cudaSuccess) {
        delete ctx;
        return CQ_ERR_NOMEM;
    }
    cudaMemsetAsync(ctx->flag.ptr, 0, 16, ctx->stream);
    cudaMemsetAsync(ctx->red_out.ptr, 0, CQ_RED_SLOTS * 8, ctx->stream);
    *out = ctx;
    return CQ_OK;
}

extern "C" void cq_ctx_destroy(cq_ctx *ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &e : ctx->ev_pool) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    for (cq_lnv *s : ctx->live_lnv) cq_lnv_detach(s);
    for (auto &kv : ctx->derived) delete kv.second;
    ctx->derived.clear();
    for (cq_pattern *p : ctx->live_patterns) {
        p->ctx = nullptr;
        for (DevBuf *b : {&p->row_ptr, &p->col, &p->row, &p->val_off, &p->transpose,
                          &p->seg_blk_dev, &p->seg_val_dev})
            b->ctx = nullptr;
        for (DevBuf *b : {&p->geo->pos, &p->geo->nb, &p->geo->cell_of, &p->geo->boxes_dev,
                          &p->geo->cell_start_dev})
            b->ctx = nullptr;
    }
    ctx->tasks.clear();
    ctx->maps.clear();
    ctx->aux.clear();
    ctx->scratch.clear();
    if (ctx->host_out) cudaFreeHost(ctx->host_out);
    delete ctx;
}

extern "C" const char *cq_last_error(const cq_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

extern "C" cq_status cq_ctx_sync(cq_ctx *ctx)
{
    if (!ctx) return CQ_ERR_INVALID;
    cq_status st = queue_flag_read(ctx);
    if (st != CQ_OK) return st;
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "stream")) != CQ_OK)
        return st;
    return check_async_flag(ctx);
}

extern "C" cq_status cq_ctx_set_mem_limit(cq_ctx *ctx, int64_t bytes)
{
    if (!ctx || bytes < 0) return CQ_ERR_INVALID;
    ctx->mem_limit = bytes;
    return CQ_OK;
}

extern "C" int64_t cq_ctx_mem_used(const cq_ctx *ctx) { return ctx ? ctx->mem_used : 0; }

// ---------------------------------------------------------------- public: patterns

extern "C" cq_status cq_pattern_build(cq_ctx *ctx, int32_t n_atoms, const double *pos_dev,
                                      const double *box_host, const int32_t *nb_dev,
                                      double range, cq_pattern **out)
{
    if (!ctx || !out) return CQ_ERR_INVALID;
    *out = nullptr;
    if (n_atoms <= 0 || !pos_dev || !box_host || !nb_dev || !(range >= 0.0) ||
        !std::isfinite(range))
        return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build: bad argument");
    for (int c = 0; c < 3; ++c)
        if (!(box_host[c] > 0.0) || !std::isfinite(box_host[c]))
            return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build: box lengths must be > 0");
    auto geo = std::make_shared<Geometry>();
    geo->id = ctx->next_id++;
    geo->device = ctx->device;
    geo->n_atoms = n_atoms;
    for (int c = 0; c < 3; ++c) geo->box[c] = box_host[c];
    geo->pos_host.resize((size_t)n_atoms * 3);
    geo->nb_host.resize(n_atoms);
    cq_status st = cq_check_cuda(ctx, cudaMemcpyAsync(geo->pos_host.data(), pos_dev,
                                                      sizeof(double) * 3 * n_atoms,
                                                      cudaMemcpyDeviceToHost, ctx->stream),
                                 "copy positions");
    if (st != CQ_OK) return st;
    st = cq_check_cuda(ctx, cudaMemcpyAsync(geo->nb_host.data(), nb_dev,
                                            sizeof(int32_t) * n_atoms,
                                            cudaMemcpyDeviceToHost, ctx->stream),
                       "copy nb");
    if (st != CQ_OK) return st;
    st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    if (st != CQ_OK) return st;
    geo->uniform_nb = geo->nb_host[0];
    for (int i = 0; i < n_atoms; ++i) {
        const int v = geo->nb_host[i];
        if (v < 1 || v > CQ_MAX_NB)
            return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build: orbitals per atom outside 1..16");
        if (v != geo->uniform_nb) geo->uniform_nb = 0;
        geo->n_orb += v;
    }
    for (size_t e = 0; e < geo->pos_host.size(); ++e)
        if (!std::isfinite(geo->pos_host[e]))
            return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build: non-finite position");
    if ((st = cq_alloc(ctx, geo->pos, sizeof(double) * 3 * n_atoms)) != CQ_OK) return st;
    if ((st = cq_alloc(ctx, geo->nb, sizeof(int32_t) * n_atoms)) != CQ_OK) return st;
    // geometry buffers outlive the context's accounting only through their patterns
    cudaMemcpyAsync(geo->pos.ptr, pos_dev, sizeof(double) * 3 * n_atoms,
                    cudaMemcpyDeviceToDevice, ctx->stream);
    cudaMemcpyAsync(geo->nb.ptr, nb_dev, sizeof(int32_t) * n_atoms, cudaMemcpyDeviceToDevice,
                    ctx->stream);
    geo->n_cells = 1;
    geo->cell_start = {0, n_atoms};
    geo->boxes.assign(box_host, box_host + 3);
    geo->cell_orb = {geo->n_orb};
    cq_pattern *p = nullptr;
    st = cq_pattern_build_geo(ctx, geo, std::vector<double>{range}, &p);
    if (st != CQ_OK) return st;
    ctx->live_patterns.push_back(p);
    *out = p;
    return CQ_OK;
}

extern "C" cq_status cq_pattern_build_batch(cq_ctx *ctx, int32_t n_cells,
                                            const int32_t *cell_start_host,
                                            const double *pos_dev, const double *boxes_host,
                                            const int32_t *nb_dev, const double *ranges_host,
                                            cq_pattern **out)
{
    if (!ctx || !out) return CQ_ERR_INVALID;
    *out = nullptr;
    if (n_cells < 1 || !cell_start_host || !boxes_host || !ranges_host || !pos_dev || !nb_dev)
        return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build_batch: bad argument");
    if (cell_start_host[0] != 0)
        return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build_batch: cell_start[0] must be 0");
    for (int c = 0; c < n_cells; ++c) {
        if (cell_start_host[c + 1] <= cell_start_host[c])
            return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build_batch: empty or unordered cell");
        if (!(ranges_host[c] >= 0.0) || !std::isfinite(ranges_host[c]))
            return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build_batch: bad range");
        for (int d = 0; d < 3; ++d)
            if (!(boxes_host[3 * c + d] > 0.0) || !std::isfinite(boxes_host[3 * c + d]))
                return cq_fail(ctx, CQ_ERR_INVALID, "pattern_build_batch: box lengths must be > 0");
    }
    const int32_t n_atoms = cell_start_host[n_cells];
    // geometry of the first cell's box for the shared fields; per-cell data below
    cq_pattern *tmp = nullptr;
    cq_status st = cq_pattern_build(ctx, n_atoms, pos_dev, boxes_host, nb_dev, 0.0, &tmp);
    if (st != CQ_OK) return st;
    std::shared_ptr<Geometry> geo = tmp->geo;
    cq_pattern_destroy(tmp);
    geo->id = ctx->next_id++;
    geo->n_cells = n_cells;
    geo->cell_start.assign(cell_start_host, cell_start_host + n_cells + 1);
    geo->boxes.assign(boxes_host, boxes_host + 3 * n_cells);
    geo->cell_orb.assign(n_cells, 0);
    std::vector<int32_t> cell_of(n_atoms);
    for (int c = 0; c < n_cells; ++c)
        for (int i = cell_start_host[c]; i < cell_start_host[c + 1]; ++i) {
            cell_of[i] = c;
            geo->cell_orb[c] += geo->nb_host[i];
        }
    if ((st = cq_alloc(ctx, geo->cell_of, sizeof(int32_t) * n_atoms)) != CQ_OK ||
        (st = cq_alloc(ctx, geo->boxes_dev, sizeof(double) * 3 * n_cells)) != CQ_OK ||
        (st = cq_alloc(ctx, geo->cell_start_dev, sizeof(int32_t) * (n_cells + 1))) != CQ_OK)
        return st;
    cudaMemcpyAsync(geo->cell_of.ptr, cell_of.data(), sizeof(int32_t) * n_atoms,
                    cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(geo->boxes_dev.ptr, geo->boxes.data(), sizeof(double) * 3 * n_cells,
                    cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(geo->cell_start_dev.ptr, geo->cell_start.data(),
                    sizeof(int32_t) * (n_cells + 1), cudaMemcpyHostToDevice, ctx->stream);
    if ((st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "batch geometry")) != CQ_OK)
        return st;
    cq_pattern *p = nullptr;
    st = cq_pattern_build_geo(ctx, geo, std::vector<double>(ranges_host, ranges_host + n_cells), &p);
    if (st != CQ_OK) return st;
    ctx->live_patterns.push_back(p);
    *out = p;
    return CQ_OK;
}

extern "C" int32_t cq_pattern_cells(const cq_pattern *p) { return p ? p->n_cells() : 0; }

extern "C" cq_status cq_pattern_info(const cq_pattern *p, int64_t *n_blocks, int64_t *n_values)
{
    if (!p) return CQ_ERR_INVALID;
    if (n_blocks) *n_blocks = p->n_blocks;
    if (n_values) *n_values = p->n_values;
    return CQ_OK;
}

extern "C" cq_status cq_pattern_export(cq_ctx *ctx, const cq_pattern *p, int64_t *row_ptr_dev,
                                       int32_t *col_dev, int64_t *val_off_dev,
                                       int64_t *transpose_dev)
{
    if (!ctx || !p) return CQ_ERR_INVALID;
    struct {
        void *dst;
        const DevBuf *src;
        size_t bytes;
    } items[4] = {
        {row_ptr_dev, &p->row_ptr, sizeof(int64_t) * (p->geo->n_atoms + 1)},
        {col_dev, &p->col, sizeof(int32_t) * p->n_blocks},
        {val_off_dev, &p->val_off, sizeof(int64_t) * p->n_blocks},
        {transpose_dev, &p->transpose, sizeof(int64_t) * p->n_blocks},
    };
    for (auto &it : items) {
        if (!it.dst || it.bytes == 0) continue;
        cq_status st = cq_check_cuda(ctx, cudaMemcpyAsync(it.dst, it.src->ptr, it.bytes,
                                                          cudaMemcpyDeviceToDevice,
                                                          ctx->stream), "export");
        if (st != CQ_OK) return st;
    }
    return CQ_OK;
}

extern "C" void cq_pattern_destroy(cq_pattern *p)
{
    if (!p || p->owned_by_ctx) return;
    cq_ctx *ctx = p->ctx;
    if (ctx) {
        cudaStreamSynchronize(ctx->stream);
        for (auto it = ctx->tasks.begin(); it != ctx->tasks.end();) {
            auto k = it->first;
            if (std::get<0>(k) == p->id || std::get<1>(k) == p->id || std::get<2>(k) == p->id)
                it = ctx->tasks.erase(it);
            else
                ++it;
        }
        for (auto it = ctx->maps.begin(); it != ctx->maps.end();) {
            auto k = it->first;
            if (std::get<0>(k) == p->id || std::get<1>(k) == p->id)
                it = ctx->maps.erase(it);
            else
                ++it;
        }
        for (auto it = ctx->aux.begin(); it != ctx->aux.end();) {
            auto k = it->first;
            if (std::get<1>(k) == p->id || std::get<2>(k) == p->id || std::get<3>(k) == p->id)
                it = ctx->aux.erase(it);
            else
                ++it;
        }
        for (size_t e = 0; e < ctx->live_patterns.size(); ++e)
            if (ctx->live_patterns[e] == p) {
                ctx->live_patterns.erase(ctx->live_patterns.begin() + e);
                break;
            }
    } else {
        // context already gone: its accounting must not be touched
        for (DevBuf *b : {&p->row_ptr, &p->col, &p->row, &p->val_off, &p->transpose}) b->ctx = nullptr;
        if (p->geo.use_count() == 1) {
            p->geo->pos.ctx = nullptr;
            p->geo->nb.ctx = nullptr;
        }
    }
    delete p;
}

// ---------------------------------------------------------------- public: products, traces

static cq_status check_triple(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                              const cq_pattern *pC)
{
    if (!pA || !pB || !pC) return cq_fail(ctx, CQ_ERR_INVALID, "null pattern");
    if (pA->ctx != ctx || pB->ctx != ctx || pC->ctx != ctx)
        return cq_fail(ctx, CQ_ERR_PATTERN, "pattern belongs to another context");
    if (!cq_same_atoms(pA, pB) || !cq_same_atoms(pA, pC))
        return cq_fail(ctx, CQ_ERR_PATTERN, "patterns over different atoms or bases");
    return CQ_OK;
}

extern "C" cq_status cq_bsmm(cq_ctx *ctx, double alpha, const cq_pattern *pA, const double *A,
                             const cq_pattern *pB, const double *B, double beta,
                             const cq_pattern *pC, double *C, cq_precision prec)
{
    if (!ctx) return CQ_ERR_INVALID;
    cq_status st = check_triple(ctx, pA, pB, pC);
    if (st != CQ_OK) return st;
    if ((!A && pA->n_values) || (!B && pB->n_values) || (!C && pC->n_values))
        return cq_fail(ctx, CQ_ERR_INVALID, "bsmm: null value array");
    if ((const double *)C == A || (const double *)C == B)
        return cq_fail(ctx, CQ_ERR_INVALID, "bsmm: C aliases an operand");
    if (!std::isfinite(alpha) || !std::isfinite(beta))
        return cq_fail(ctx, CQ_ERR_INVALID, "bsmm: non-finite alpha/beta");
    if (prec != CQ_FP64 && prec != CQ_SPLIT_BF16X3 && prec != CQ_FP64_EMU)
        return cq_fail(ctx, CQ_ERR_INVALID, "bsmm: unknown precision");
    TaskList *tl = nullptr;
    if ((st = cq_get_tasks(ctx, pA, pB, pC, &tl)) != CQ_OK) return st;
    if (prec == CQ_FP64) return cq_bsmm_f64(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
    if (prec == CQ_FP64_EMU) return cq_bsmm_emu(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
    return cq_bsmm_split(ctx, tl, alpha, pA, A, pB, B, beta, pC, C);
}

extern "C" cq_status cq_bsmm_work(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                                  const cq_pattern *pC, int64_t *triplets_host,
                                  double *flops_host)
{
    if (!ctx) return CQ_ERR_INVALID;
    cq_status st = check_triple(ctx, pA, pB, pC);
    if (st != CQ_OK) return st;
    TaskList *tl = nullptr;
    if ((st = cq_get_tasks(ctx, pA, pB, pC, &tl)) != CQ_OK) return st;
    if (triplets_host) *triplets_host = tl->n_tasks;
    if (flops_host) *flops_host = tl->flops;
    return CQ_OK;
}

extern "C" cq_status cq_bsmm_config(cq_ctx *ctx, const cq_pattern *pA, const cq_pattern *pB,
                                    const cq_pattern *pC, int32_t *lane_split_host,
                                    int32_t *tuned_host)
{
    if (!ctx) return CQ_ERR_INVALID;
    cq_status st = check_triple(ctx, pA, pB, pC);
    if (st != CQ_OK) return st;
    TaskList *tl = nullptr;
    if ((st = cq_get_tasks(ctx, pA, pB, pC, &tl)) != CQ_OK) return st;
    if (lane_split_host) *lane_split_host = cq_lane_split(tl);
    if (tuned_host) *tuned_host = tl->q != 0;
    return CQ_OK;
}

extern "C" cq_status cq_trace_prod(cq_ctx *ctx, const cq_pattern *pA, const double *A,
                                   const cq_pattern *pB, const double *B, double *out_host)
{
    if (!ctx || !out_host) return CQ_ERR_INVALID;
    cq_status st = check_triple(ctx, pA, pB, pB);
    if (st != CQ_OK) return st;
    if ((st = cq_trace_dev(ctx, pA, A, pB, B, 0)) != CQ_OK) return st;
    return cq_fetch(ctx, 0, 1, out_host);
}

extern "C" cq_status cq_dot(cq_ctx *ctx, const cq_pattern *p, const double *A, const double *B,
                            double *out_host)
{
    if (!ctx || !p || !out_host) return CQ_ERR_INVALID;
    if (p->ctx != ctx) return cq_fail(ctx, CQ_ERR_PATTERN, "pattern of another context");
    cq_status st = cq_dot_dev(ctx, p, A, B, 0);
    if (st != CQ_OK) return st;
    return cq_fetch(ctx, 0, 1, out_host);
}

// ---------------------------------------------------------------- timing and FP64 peak

void cq_timing_begin(cq_ctx *ctx, double flops, double mma_flops)
{
    if (!ctx->timing || ctx->capturing) return;
    ctx->timed_mma_flops += mma_flops;
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        ctx->ev_pool.push_back({a, b});
    }
    cudaEventRecord(ctx->ev_pool[ctx->ev_used].first, ctx->stream);
    ctx->timed_flops += flops;
}

void cq_timing_end(cq_ctx *ctx)
{
    if (!ctx->timing || ctx->capturing) return;
    cudaEventRecord(ctx->ev_pool[ctx->ev_used].second, ctx->stream);
    ctx->ev_used++;
}

extern "C" cq_status cq_ctx_set_timing(cq_ctx *ctx, int on)
{
    if (!ctx) return CQ_ERR_INVALID;
    ctx->timing = on != 0;
    return CQ_OK;
}

extern "C" cq_status cq_ctx_set_autotune(cq_ctx *ctx, int on)
{
    if (!ctx) return CQ_ERR_INVALID;
    ctx->autotune = on != 0;
    return CQ_OK;
}

extern "C" cq_status cq_ctx_set_graphs(cq_ctx *ctx, int on)
{
    if (!ctx) return CQ_ERR_INVALID;
    if (on && ctx->stream == nullptr)
        return cq_fail(ctx, CQ_ERR_INVALID,
                       "graphs need a context on a created stream (the default stream cannot be captured)");
    ctx->graphs = on != 0;
    return CQ_OK;
}

extern "C" cq_status cq_ctx_release_cache(cq_ctx *ctx)
{
    if (!ctx) return CQ_ERR_INVALID;
    if (ctx->capturing) return cq_fail(ctx, CQ_ERR_INVALID, "release_cache inside a graph capture");
    cq_status st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "release cache");
    if (st != CQ_OK) return st;
    ctx->tasks.clear();
    ctx->maps.clear();
    ctx->aux.clear();
    ctx->scratch.clear();
    ctx->scratch_gen++;  // captured graphs name the freed buffers: capture them again
    return CQ_OK;
}

extern "C" cq_status cq_ctx_set_test_wait(cq_ctx *ctx, int64_t cycles)
{
    if (!ctx || cycles < 0 || cycles > 100000000) return CQ_ERR_INVALID;
    ctx->test_wait_cycles = cycles;
    return CQ_OK;
}

extern "C" cq_status cq_ctx_kernel_stats(cq_ctx *ctx, int64_t *launches_host, double *ms_host,
                                         double *flops_host, double *mma_flops_host)
{
    if (!ctx) return CQ_ERR_INVALID;
    cq_status st = cq_check_cuda(ctx, cudaStreamSynchronize(ctx->stream), "sync");
    if (st != CQ_OK) return st;
    double ms = 0.0;
    for (size_t e = 0; e < ctx->ev_used; ++e) {
        float t = 0.f;
        st = cq_check_cuda(ctx, cudaEventElapsedTime(&t, ctx->ev_pool[e].first,
                                                     ctx->ev_pool[e].second), "event time");
        if (st != CQ_OK) return st;
        ms += t;
    }
    if (launches_host) *launches_host = (int64_t)ctx->ev_used;
    if (ms_host) *ms_host = ms;
    if (flops_host) *flops_host = ctx->timed_flops;
    if (mma_flops_host) *mma_flops_host = ctx->timed_mma_flops;
    ctx->timed_mma_flops = 0.0;
    ctx->ev_used = 0;
    ctx->timed_flops = 0.0;
    return CQ_OK;
}

namespace {
__global__ void k_fp64_fma_chain(int iters, double seed, double *sink)
{
    double a[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) a[e] = seed + threadIdx.x * 1e-9 + e;
    const double m = 0.999999999, c = 1e-12;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = fma(a[e], m, c);
    }
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < 8; ++e) s += a[e];
    if (s == 12345.678) sink[0] = s;  // keeps the chain live; never true in practice
}

// The same on the FP64 tensor path: independent m8n8k4 DMMA chains (512 flops each).
__global__ void k_fp64_dmma_chain(int iters, double seed, double *sink)
{
    const double a = seed + threadIdx.x * 1e-9, b = 0.5;
    double c[4][2];
#pragma unroll
    for (int e = 0; e < 4; ++e) c[e][0] = c[e][1] = 0.0;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int e = 0; e < 4; ++e)
            asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, "
                         "{%0,%1};"
                         : "+d"(c[e][0]), "+d"(c[e][1])
                         : "d"(a), "d"(b));
    }
    double s = 0.0;
#pragma unroll
    for (int e = 0; e < 4; ++e) s += c[e][0] + c[e][1];
    if (s == 12345.678) sink[0] = s;
}
}  // namespace

extern "C" cq_status cq_peak_fp64(cq_ctx *ctx, double *flops_per_s_host)
{
    if (!ctx || !flops_per_s_host) return CQ_ERR_INVALID;
    // Best of the FMA path and the DMMA path, each timed over ~1 s after a warm-up launch.
    const int blocks = ctx->num_sms * 8, threads = 256, iters = 4096, reps = 5;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    double *sink = ctx->red_out.as<double>() + 63;
    double best = 0.0;
    cq_status st = CQ_OK;
    for (int kind = 0; kind < 2 && st == CQ_OK; ++kind) {
        const int it = kind == 0 ? iters : iters / 4;
        auto launch = [&](double seed) {
            if (kind == 0)
                k_fp64_fma_chain<<<blocks, threads, 0, ctx->stream>>>(it, seed, sink);
            else
                k_fp64_dmma_chain<<<blocks, threads, 0, ctx->stream>>>(it, seed, sink);
        };
        launch(1.0);
        cudaEventRecord(a, ctx->stream);
        for (int r = 0; r < reps; ++r) launch(1.0 + r);
        cudaEventRecord(b, ctx->stream);
        cq_count_launch(reps + 1);
        st = cq_check_cuda(ctx, cudaEventSynchronize(b), "fp64 probe");
        float ms = 0.f;
        if (st == CQ_OK) cudaEventElapsedTime(&ms, a, b);
        const double per_thread = kind == 0 ? 2.0 * 8.0 * it : 512.0 * 4.0 * it / 32.0;
        const double flops = per_thread * (double)blocks * threads * reps;
        if (ms > 0.f) best = std::max(best, flops / (ms * 1e-3));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (st != CQ_OK) return st;
    *flops_per_s_host = best;
    return CQ_OK;
}
