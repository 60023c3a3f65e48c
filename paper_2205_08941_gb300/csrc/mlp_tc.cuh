// Tensor-core GEMM of the learned-guess network (included by guess.cu): C = A Bt^T with BF16
// operands and FP32 accumulation in tensor memory (tcgen05.mma kind::f16), for the three
// contractions of the MLP -- the forward layer Z = H W, the backward dH = dZ W^T and the
// weight gradient dW = H^T dZ (from transposed BF16 copies of H and dZ).
//
// C[m][n] = sum_{k in the CTA's K range} A[m][k] Bt[n][k] for m < M, n < N.  A (M x K) and
// Bt (N x K) are row-major BF16 with leading dimensions lda, ldb (elements).  One CTA of 128
// threads owns 128 rows and 64 columns of C (blockIdx.y picks the column tile; one MMA of the
// tile's width rounded up to 16); K runs in chunks of up to 256 staged in shared memory in
// the canonical no-swizzle K-major layout (core matrices of 8 rows x 16 bytes, adjacent
// along K, 8-row groups 4 KB apart); two CTAs fit one SM.  Blocks along z take consecutive K ranges of k_chunk and write their own partial
// C (c_stride_z apart), summed later in a fixed order, so results are deterministic.
//
// The MMA completion wait is bounded (about two seconds); a CTA that gives up sets bit 16
// of the flag word, frees its tensor memory and returns.
constexpr int TC_MT = 128;      // rows of C per CTA
constexpr int TC_NT = 64;       // columns of C per CTA
constexpr int TC_KC = 256;      // K values per staged chunk
constexpr int TC_SBO = (TC_KC / 8) * 128;
constexpr int TC_SMEM = TC_MT * TC_KC * 2 + TC_NT * TC_KC * 2 + 64;
constexpr long long TC_WAIT = 4000000000LL;

__device__ __forceinline__ uint32_t tc_smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)(128 >> 4) << 16;
    d |= (uint64_t)(TC_SBO >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// rows [r0, r0 + rows) of a row-major BF16 matrix, K range [k0, k0 + kn), into the staged
// layout (zeros outside the matrix or the range); kn16 = kn rounded up to 16
__device__ __forceinline__ void tc_stage(uint8_t *dst, int rows, const __nv_bfloat16 *src,
                                         int64_t ld, int r0, int rmax, int64_t k0, int64_t kend,
                                         int kn16)
{
    const int groups = kn16 / 8;
    for (int e = threadIdx.x; e < rows * groups; e += blockDim.x) {
        const int r = e / groups, g = e % groups;
        const int64_t k = k0 + 8 * g;
        uint4 w = make_uint4(0u, 0u, 0u, 0u);
        if (r0 + r < rmax) {
            const __nv_bfloat16 *p = src + (int64_t)(r0 + r) * ld + k;
            if (k + 8 <= kend && (reinterpret_cast<uintptr_t>(p) & 15) == 0) {
                w = __ldg(reinterpret_cast<const uint4 *>(p));  // eight values in one load
            } else {
                uint32_t u[4] = {0u, 0u, 0u, 0u};
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (k + q < kend)
                        u[q >> 1] |= (uint32_t)__bfloat16_as_ushort(p[q]) << (16 * (q & 1));
                w = make_uint4(u[0], u[1], u[2], u[3]);
            }
        }
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * TC_SBO + g * 128 + (r & 7) * 16) = w;
    }
}

__global__ void __launch_bounds__(128, 2)
k_gemm_tc(int M, int N, const __nv_bfloat16 *A, int64_t lda, const __nv_bfloat16 *Bt,
          int64_t ldb, float *C, int64_t ldc, int64_t k0, int64_t k1, int64_t c_stride_z,
          int64_t k_chunk, int32_t *flag)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t *sa = smem, *sb = smem + TC_MT * TC_KC * 2;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb + TC_NT * TC_KC * 2);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem_u32(bar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         tc_smem_u32(tslot)),
                     "r"(TC_NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const int m0 = blockIdx.x * TC_MT, n0 = blockIdx.y * TC_NT;
    const int Npad = ((min(TC_NT, N - n0) + 15) / 16) * 16;  // this tile's MMA width
    const int64_t kb = k0 + (int64_t)blockIdx.z * k_chunk;
    const int64_t ke = min(k1, kb + k_chunk);
    // kind::f16: D = F32, A = B = BF16, both K-major, N = Npad, M = 128
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Npad >> 3) << 17) |
                           ((uint32_t)(TC_MT >> 4) << 24);
    uint32_t phase = 0;
    bool issued = false, ok = true;
    for (int64_t kc = kb; kc < ke && ok; kc += TC_KC) {
        const int kn = (int)min((int64_t)TC_KC, ke - kc);
        const int kn16 = (kn + 15) & ~15;
        tc_stage(sa, TC_MT, A, lda, m0, M, kc, ke, kn16);
        tc_stage(sb, Npad, Bt, ldb, n0, N, kc, ke, kn16);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint64_t da = tc_desc(tc_smem_u32(sa)), db = tc_desc(tc_smem_u32(sb));
            for (int ks = 0; ks < kn16 / 16; ++ks) {
                const uint32_t acc = (issued || ks > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                    "l"(da + (uint64_t)((ks * 256) >> 4)), "l"(db + (uint64_t)((ks * 256) >> 4)),
                    "r"(idesc), "r"(acc));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    tc_smem_u32(bar))
                : "memory");
        }
        issued = true;
        // every thread waits for the chunk's MMAs before the next staging overwrites them;
        // past the limit the call has failed, but the wait goes on (bounded again) so that
        // no MMA is still writing when the tensor memory is freed
        const long long t0 = clock64();
        for (;;) {
            uint32_t done;
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(tc_smem_u32(bar)), "r"(phase)
                : "memory");
            if (done) break;
            const long long dt = clock64() - t0;
            if (dt > TC_WAIT) ok = false;
            if (dt > 2 * TC_WAIT) break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        ok = __syncthreads_and(ok);  // uniform: every thread leaves the loop together
    }
    if (ok) {
        // epilogue: warp w holds rows m0 + 32 w + lane of the accumulator
        const int row = m0 + warp * 32 + lane;
        float *Cz = C + (int64_t)blockIdx.z * c_stride_z;
        for (int cb = 0; cb < Npad; cb += 16) {
            uint32_t v[16];
            if (issued) {
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,"
                    "%11,%12,%13,%14,%15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                    : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            } else {
#pragma unroll
                for (int x = 0; x < 16; ++x) v[x] = 0u;
            }
            if (row < M) {
#pragma unroll
                for (int x = 0; x < 16; ++x)
                    if (n0 + cb + x < N) Cz[(int64_t)row * ldc + n0 + cb + x] = __uint_as_float(v[x]);
            }
        }
    } else if (t == 0) {
        atomicOr(flag, 16);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_NT));
    }
}

// BF16 copy of a row-major FP32 matrix (rows x cols), optionally transposed into a
// cols x ld_t matrix (ld_t >= rows; columns rows.. ld_t - 1 are left as they are).
__global__ void k_to_bf16_mat(int64_t rows, int cols, const float *src, __nv_bfloat16 *dst,
                              int transpose, int64_t ld_t)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= rows * cols) return;
    const int64_t r = e / cols;
    const int c = (int)(e % cols);
    const __nv_bfloat16 v = __float2bfloat16(src[e]);
    if (transpose)
        dst[(int64_t)c * ld_t + r] = v;
    else
        dst[e] = v;
}

// Transposed BF16 copy of a row-major FP32 matrix (rows x cols) into a cols x ld_t matrix,
// through 32 x 32 shared-memory tiles so that reads and writes both run along rows (one CTA
// of 32 x 8 threads per tile).
__global__ void __launch_bounds__(256)
k_to_bf16_t(int64_t rows, int cols, const float *src, __nv_bfloat16 *dst, int64_t ld_t)
{
    __shared__ float tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32;
    const int c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int64_t r = r0 + y;
        const int c = c0 + threadIdx.x;
        tile[y][threadIdx.x] = (r < rows && c < cols) ? src[r * cols + c] : 0.f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) {
        const int c = c0 + y;
        const int64_t r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[(int64_t)c * ld_t + r] = __float2bfloat16(tile[threadIdx.x][y]);
    }
}
