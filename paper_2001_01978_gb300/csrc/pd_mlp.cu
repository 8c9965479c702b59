// pd_mlp.cu -- the learned Lanczos warm start.
//
// A small network maps per-orbit features of a problem (e, G, N) to one weight
// w_i per orbit; the start vector is psi(s) = exp(sum_{i in s} w_i), a product
// over the occupied orbits of each basis state (the form of a number-projected
// BCS state, which is close to the exact pairing ground state).  Training
// targets come from ground states computed by this solver: for each training
// problem, w* minimises sum_s psi(s)^2 (log|psi(s)| - sum_{i in s} w_i)^2.
//
// Network: 16 -> 128 -> 128 -> 128 -> 1, SiLU, bfloat16 operands with FP32
// accumulation on the tensor cores (tcgen05.mma, accumulators in tensor
// memory), FP32 master weights, Adam.  Sizes are tiny (rows = orbits of the
// training problems), so one tiled kernel serves every product of the forward
// and backward passes.
#include "pd_internal.h"
#include "pairdiag.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

using namespace pd;

namespace {

constexpr int kF = 16, kH = 128;
constexpr int oW1 = 0, ob1 = oW1 + kF * kH, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH * kH, ow4 = ob3 + kH, ob4 = ow4 + kH, kNParams = ob4 + 1;

using bf16 = __nv_bfloat16;

// ---- C[M,128] (=, or += over split K) op(A)[M,K] op(B)[K,128] on the 5th-generation
// tensor cores: tcgen05.mma with bfloat16 operands in shared memory and an FP32
// accumulator in tensor memory (TMEM).
// A(m,k) = TA ? A[k*lda + m] : A[m*lda + k];  B(k,n) = TB ? B[n*ldb + k] : B[k*ldb + n].
// Every product of the network has N = 128 (the layer width).  One CTA of 128
// threads computes a 128 x 128 tile of C over a range of K (split K over
// gridDim.y, added with atomics into a zeroed C):
//   - the four warps stage a 128 x 64 slice of A and of B^T in shared memory in
//     the canonical K-major layout without swizzle: 8 x 16-byte core matrices,
//     element (r, k) at (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2
//     bytes, so the leading (K) byte offset of the descriptor is 128 and the
//     stride (8-row) byte offset 1024;
//   - one thread issues four tcgen05.mma (M = N = 128, K = 16 each) into the
//     TMEM accumulator (128 lanes = rows of C, 128 columns) and commits them
//     to an mbarrier, which every thread waits on before the slice is
//     overwritten;
//   - the epilogue reads the accumulator with tcgen05.ld (each warp its 32
//     lanes) and writes C.
// Waits are bounded: on expiry the kernel sets *err, still frees its TMEM and
// returns (the caller reports PD_ETIMEOUT).  The network's products are tiny
// (M = the orbit rows of the problems, K <= rows), so staging by threads
// instead of TMA is no bottleneck.
constexpr int kTileM = 128, kTileN = 128, kSliceK = 64;
constexpr int kTmemCols = 128;                 // one FP32 column per output column
constexpr long long kSpinLimit = 1ll << 26;    // mbarrier polls before giving up
constexpr int kGemmPadSmem = 18 * 1024;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared memory matrix descriptor: K-major, no swizzle
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);            // start address
    d |= (uint64_t)((128u & 0x3FFFFu) >> 4) << 16;        // leading (K) byte offset: next core matrix in K
    d |= (uint64_t)((1024u & 0x3FFFFu) >> 4) << 32;       // stride byte offset: next 8 rows
    d |= (uint64_t)1 << 46;                               // descriptor version of this architecture
    return d;                                             // base offset 0, no swizzle
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = 128, M = 128
constexpr uint32_t kIdescBf16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                                ((uint32_t)(kTileM >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase)
{
    for (long long it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(bar), "r"(phase)
                     : "memory");
        if (done) return true;
    }
    return false;
}

// stage rows [r0, r0 + 128) x k [k0, k0 + 64) of op(X) (row index r, column k)
// into the canonical layout; zero outside [0, nrow) x [k0, kend)
template <bool TR>
__device__ __forceinline__ void stage_slice(unsigned char *dst, const bf16 *__restrict__ X, int ld, int r0, int nrow,
                                            int k0, int kend)
{
    const bf16 zero = __float2bfloat16(0.0f);
    for (int it = threadIdx.x; it < kTileM * (kSliceK / 8); it += blockDim.x) {
        const int r = it % kTileM, kc = it / kTileM;        // consecutive threads: consecutive rows
        const int gr = r0 + r;
        __align__(16) bf16 v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int gk = k0 + kc * 8 + j;
            v[j] = (gr < nrow && gk < kend) ? (TR ? X[(size_t)gk * ld + gr] : X[(size_t)gr * ld + gk]) : zero;
        }
        *reinterpret_cast<uint4 *>(dst + (r >> 3) * 1024 + kc * 128 + (r & 7) * 16) =
            *reinterpret_cast<const uint4 *>(v);
    }
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(128)
gemm_tc_kernel(int M, int K, const bf16 *__restrict__ A, int lda, const bf16 *__restrict__ B, int ldb,
               float *__restrict__ C, int ldc, int *err)
{
    __shared__ __align__(1024) unsigned char sA[kTileM * kSliceK * 2];
    __shared__ __align__(1024) unsigned char sB[kTileN * kSliceK * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * kTileM;
    const int kchunk = ((K + gridDim.y - 1) / gridDim.y + kSliceK - 1) / kSliceK * kSliceK;
    const int kbeg = blockIdx.y * kchunk, kend = min(K, kbeg + kchunk);
    if (kbeg >= kend) return;                          // CTA-uniform: nothing to add
    const bool split = gridDim.y > 1;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = s_tmem;
    const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB), barp = smem_u32(&bar);

    uint32_t phase = 0;
    bool timed_out = false;
    for (int k0 = kbeg; k0 < kend && !timed_out; k0 += kSliceK) {
        stage_slice<TA>(sA, A, lda, m0, M, k0, kend);
        stage_slice<!TB>(sB, B, ldb, 0, kTileN, k0, kend);   // row n of B^T: B(k, n)
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");   // generic-proxy stores -> async proxy
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (int sk = 0; sk < kSliceK / 16; ++sk) {
                const uint64_t da = umma_desc(a0 + sk * 256), db = umma_desc(b0 + sk * 256);
                const uint32_t accum = (k0 == kbeg && sk == 0) ? 0u : 1u;
                asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
                             "l"(da), "l"(db), "r"(kIdescBf16), "r"(accum)
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(barp)
                         : "memory");
        }
        // the slice may be overwritten only after these MMAs have read it
        const bool ok = mbar_wait(barp, phase);
        phase ^= 1u;
        timed_out = __syncthreads_or(!ok) != 0;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (timed_out) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w + 31
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < kTileN; c0 += 32) {
            uint32_t v[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
                         "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
                         "%28, %29, %30, %31}, [%32];\n"
                         : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                           "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                           "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
                           "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
                           "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                         : "r"(taddr)
                         : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (row < M) {
                float *dst = C + (size_t)row * ldc + c0;
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float f = __uint_as_float(v[j]);
                    if (split) atomicAdd(dst + j, f);
                    else dst[j] = f;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// C[M, 128] = op(A) op(B) (split K over ksplit CTAs per row tile, C zeroed first)
template <bool TA, bool TB>
void gemm(int M, int N, int K, const bf16 *A, int lda, const bf16 *B, int ldb, float *C, int ldc, int ksplit,
          int *err, cudaStream_t st)
{
    (void)N;                                   // always kTileN (the layer width)
    dim3 grid((M + kTileM - 1) / kTileM, ksplit);
    if (ksplit > 1) cudaMemsetAsync(C, 0, sizeof(float) * (size_t)M * ldc, st);
    // 18 KB of unused dynamic shared memory keep at most four CTAs on an SM,
    // so their 4 x 128 TMEM columns fit the SM's 512 and no allocation waits
    static const cudaError_t attr =       // static + dynamic shared memory above 48 KB needs the opt-in
        cudaFuncSetAttribute(gemm_tc_kernel<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmPadSmem);
    (void)attr;
    gemm_tc_kernel<TA, TB><<<grid, 128, kGemmPadSmem, st>>>(M, K, A, lda, B, ldb, C, ldc, err);
    count_launches(1);
}

// ---- elementwise pieces ------------------------------------------------------
__device__ __forceinline__ float silu(float z) { return z / (1.0f + __expf(-z)); }
__device__ __forceinline__ float dsilu(float z)
{
    const float s = 1.0f / (1.0f + __expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// Z += bias (in place, FP32), A = silu(Z) in bfloat16
__global__ void bias_silu_kernel(float *__restrict__ Z, const float *__restrict__ bias, bf16 *__restrict__ Aout,
                                 int rows)
{
    const int64_t n = (int64_t)rows * kH;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float z = Z[i] + bias[i % kH];
        Z[i] = z;
        Aout[i] = __float2bfloat16(silu(z));
    }
}

// out[r] = A3[r,:] . w4 + b4 (one warp per row)
__global__ void head_kernel(const bf16 *__restrict__ A3, const bf16 *__restrict__ w4, const float *__restrict__ b4,
                            float *__restrict__ out, int rows)
{
    const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (r >= rows) return;
    float s = 0.0f;
    for (int j = lane; j < kH; j += 32) s += __bfloat162float(A3[(size_t)r * kH + j]) * __bfloat162float(w4[j]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s + b4[0];
}

// dout = 2 (out - t) / rows; loss partial sums
__global__ void loss_kernel(const float *__restrict__ out, const float *__restrict__ t, float *__restrict__ dout,
                            int rows, double *__restrict__ loss)
{
    __shared__ double sh[256];
    double acc = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += gridDim.x * blockDim.x) {
        const float d = out[r] - t[r];
        dout[r] = 2.0f * d / (float)rows;
        acc += (double)d * d;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, sh[0] / rows);
}

// head backward: g_w4[j] = sum_r A3[r,j] dout[r], g_b4 = sum dout; dZ3 = dout w4 silu'(Z3)
__global__ void head_back_kernel(const bf16 *__restrict__ A3, const float *__restrict__ Z3, const bf16 *__restrict__ w4,
                                 const float *__restrict__ dout, int rows, float *__restrict__ gw4,
                                 float *__restrict__ gb4, bf16 *__restrict__ dZ, float *__restrict__ gb3)
{
    const int j = threadIdx.x;                 // column (blockDim.x == kH)
    float sw = 0.0f, sb = 0.0f, sz = 0.0f;
    const float wj = __bfloat162float(w4[j]);
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const float d = dout[r];
        const size_t i = (size_t)r * kH + j;
        sw += __bfloat162float(A3[i]) * d;
        if (j == 0) sb += d;
        const float dz = d * wj * dsilu(Z3[i]);
        dZ[i] = __float2bfloat16(dz);
        sz += dz;
    }
    atomicAdd(&gw4[j], sw);
    atomicAdd(&gb3[j], sz);
    if (j == 0) atomicAdd(gb4, sb);
}

// dZ = dA silu'(Z) (dA FP32 from a product), bias gradient column sums
__global__ void dsilu_kernel(const float *__restrict__ dA, const float *__restrict__ Z, int rows,
                             bf16 *__restrict__ dZ, float *__restrict__ gb)
{
    const int j = threadIdx.x;
    float sz = 0.0f;
    for (int r = blockIdx.x; r < rows; r += gridDim.x) {
        const size_t i = (size_t)r * kH + j;
        const float dz = dA[i] * dsilu(Z[i]);
        dZ[i] = __float2bfloat16(dz);
        sz += dz;
    }
    atomicAdd(&gb[j], sz);
}

__global__ void to_bf16_kernel(const float *__restrict__ src, bf16 *__restrict__ dst, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = __float2bfloat16(src[i]);
}

__global__ void adam_kernel(float *__restrict__ th, const float *__restrict__ g, float *__restrict__ m1,
                            float *__restrict__ m2, int n, float lr, float b1, float b2, float c1, float c2, float eps)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float a = b1 * m1[i] + (1.0f - b1) * gi;
        const float v = b2 * m2[i] + (1.0f - b2) * gi * gi;
        m1[i] = a;
        m2[i] = v;
        th[i] -= lr * (a / c1) / (sqrtf(v / c2) + eps);
    }
}

}  // namespace

// ---- the network handle ----------------------------------------------------------
struct pairdiag_mlp {
    float *theta = nullptr;      // FP32 master parameters
    bf16 *wb = nullptr;          // bfloat16 copies (same layout)
    float *grad = nullptr, *m1 = nullptr, *m2 = nullptr;
    int cap = 0;                 // rows the work buffers hold
    bf16 *X = nullptr, *A1 = nullptr, *A2 = nullptr, *A3 = nullptr;
    bf16 *dZ1 = nullptr, *dZ2 = nullptr, *dZ3 = nullptr;   // backward intermediates, one per layer
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *dA1 = nullptr, *dA2 = nullptr;
    float *out = nullptr, *t = nullptr, *dout = nullptr;
    int *err = nullptr;          // set by a tensor-core product whose bounded wait expired
    double *loss = nullptr;
    int steps = 0;
    cudaStream_t st = nullptr;
};

namespace {

void mlp_free_work(pairdiag_mlp *m)
{
    void *p[] = {m->X, m->A1, m->A2, m->A3, m->dZ1, m->dZ2, m->dZ3, m->Z1, m->Z2, m->Z3, m->dA1, m->dA2,
                 m->out, m->t, m->dout};
    for (void *q : p)
        if (q) cudaFree(q);
    m->X = m->A1 = m->A2 = m->A3 = m->dZ1 = m->dZ2 = m->dZ3 = nullptr;
    m->Z1 = m->Z2 = m->Z3 = m->dA1 = m->dA2 = m->out = m->t = m->dout = nullptr;
    m->cap = 0;
}

int mlp_reserve(pairdiag_mlp *m, int rows)
{
    if (rows <= m->cap) return PD_OK;
    mlp_free_work(m);
    const size_t nh = (size_t)rows * kH;
    PD_CUDA(cudaMalloc(&m->X, sizeof(bf16) * (size_t)rows * kF));
    PD_CUDA(cudaMalloc(&m->A1, sizeof(bf16) * nh));
    PD_CUDA(cudaMalloc(&m->A2, sizeof(bf16) * nh));
    PD_CUDA(cudaMalloc(&m->A3, sizeof(bf16) * nh));
    PD_CUDA(cudaMalloc(&m->dZ1, sizeof(bf16) * nh));
    PD_CUDA(cudaMalloc(&m->dZ2, sizeof(bf16) * nh));
    PD_CUDA(cudaMalloc(&m->dZ3, sizeof(bf16) * nh));
    PD_CUDA(cudaMalloc(&m->Z1, sizeof(float) * nh));
    PD_CUDA(cudaMalloc(&m->Z2, sizeof(float) * nh));
    PD_CUDA(cudaMalloc(&m->Z3, sizeof(float) * nh));
    PD_CUDA(cudaMalloc(&m->dA1, sizeof(float) * nh));
    PD_CUDA(cudaMalloc(&m->dA2, sizeof(float) * nh));
    PD_CUDA(cudaMalloc(&m->out, sizeof(float) * rows));
    PD_CUDA(cudaMalloc(&m->t, sizeof(float) * rows));
    PD_CUDA(cudaMalloc(&m->dout, sizeof(float) * rows));
    m->cap = rows;
    return PD_OK;
}

int grid1(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, sm_count() * 8)); }

// after a synchronisation of m->st: PD_ETIMEOUT (and the flag cleared) when a
// tensor-core product gave up waiting for its MMAs
int check_tc(pairdiag_mlp *m)
{
    int e = 0;
    PD_CUDA(cudaMemcpy(&e, m->err, sizeof e, cudaMemcpyDeviceToHost));
    if (e) {
        PD_CUDA(cudaMemset(m->err, 0, sizeof e));
        return fail(PD_ETIMEOUT, "mlp: a tensor-core product timed out waiting for its MMAs");
    }
    return PD_OK;
}

// forward pass on m->X (rows x 16, bfloat16) -> m->out
int mlp_forward(pairdiag_mlp *m, int rows)
{
    cudaStream_t st = m->st;
    to_bf16_kernel<<<grid1(kNParams), 256, 0, st>>>(m->theta, m->wb, kNParams);
    gemm<false, false>(rows, kH, kF, m->X, kF, m->wb + oW1, kH, m->Z1, kH, 1, m->err, st);
    bias_silu_kernel<<<grid1((int64_t)rows * kH), 256, 0, st>>>(m->Z1, m->theta + ob1, m->A1, rows);
    gemm<false, false>(rows, kH, kH, m->A1, kH, m->wb + oW2, kH, m->Z2, kH, 1, m->err, st);
    bias_silu_kernel<<<grid1((int64_t)rows * kH), 256, 0, st>>>(m->Z2, m->theta + ob2, m->A2, rows);
    gemm<false, false>(rows, kH, kH, m->A2, kH, m->wb + oW3, kH, m->Z3, kH, 1, m->err, st);
    bias_silu_kernel<<<grid1((int64_t)rows * kH), 256, 0, st>>>(m->Z3, m->theta + ob3, m->A3, rows);
    head_kernel<<<(rows * 32 + 255) / 256, 256, 0, st>>>(m->A3, m->wb + ow4, m->theta + ob4, m->out, rows);
    count_launches(5);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// loss and gradient (after mlp_forward) -> m->grad, m->loss
int mlp_backward(pairdiag_mlp *m, int rows)
{
    cudaStream_t st = m->st;
    const int ks = std::max(1, std::min(64, rows / 256));
    PD_CUDA(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNParams, st));
    PD_CUDA(cudaMemsetAsync(m->loss, 0, sizeof(double), st));
    loss_kernel<<<std::max(1, std::min(64, (rows + 255) / 256)), 256, 0, st>>>(m->out, m->t, m->dout, rows, m->loss);
    const int gr = std::max(1, std::min(1024, rows));
    head_back_kernel<<<gr, kH, 0, st>>>(m->A3, m->Z3, m->wb + ow4, m->dout, rows, m->grad + ow4, m->grad + ob4,
                                        m->dZ3, m->grad + ob3);
    // layer 3: gW3 = A2^T dZ3 (written straight into the gradient), dA2 = dZ3 W3^T
    gemm<true, false>(kH, kH, rows, m->A2, kH, m->dZ3, kH, m->grad + oW3, kH, ks, m->err, st);
    gemm<false, true>(rows, kH, kH, m->dZ3, kH, m->wb + oW3, kH, m->dA2, kH, 1, m->err, st);
    dsilu_kernel<<<gr, kH, 0, st>>>(m->dA2, m->Z2, rows, m->dZ2, m->grad + ob2);
    // layer 2
    gemm<true, false>(kH, kH, rows, m->A1, kH, m->dZ2, kH, m->grad + oW2, kH, ks, m->err, st);
    gemm<false, true>(rows, kH, kH, m->dZ2, kH, m->wb + oW2, kH, m->dA1, kH, 1, m->err, st);
    dsilu_kernel<<<gr, kH, 0, st>>>(m->dA1, m->Z1, rows, m->dZ1, m->grad + ob1);
    // layer 1: gW1 = X^T dZ1
    gemm<true, false>(kF, kH, rows, m->X, kF, m->dZ1, kH, m->grad + oW1, kH, ks, m->err, st);
    count_launches(4);
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

int mlp_load_inputs(pairdiag_mlp *m, int rows, const float *X, const float *t)
{
    PD_TRY(mlp_reserve(m, rows));
    std::vector<bf16> xb((size_t)rows * kF);
    for (size_t i = 0; i < xb.size(); ++i) xb[i] = __float2bfloat16(X[i]);
    PD_CUDA(cudaMemcpyAsync(m->X, xb.data(), sizeof(bf16) * xb.size(), cudaMemcpyHostToDevice, m->st));
    if (t) PD_CUDA(cudaMemcpyAsync(m->t, t, sizeof(float) * rows, cudaMemcpyHostToDevice, m->st));
    PD_CUDA(cudaStreamSynchronize(m->st));          // host staging buffers go out of scope
    return PD_OK;
}

// ---- start vector and target fit over the basis blocks ---------------------------
// v[s] = exp(sum_{p in s} w_p - shift)
struct OrbitWeights {                   // per-orbit weights, passed by value (no device allocation)
    double w[kMaxOmega];
};

template <typename T>
__global__ void __launch_bounds__(256)
product_start_kernel(const Blocks B, const OrbitWeights w, double shift, T *__restrict__ v)
{
    __shared__ double sw[kMaxOmega];
    for (int p = threadIdx.x; p < B.omega; p += blockDim.x) sw[p] = w.w[p];
    __syncthreads();
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b], base = B.blk_base[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        int off = 0;
        for (int j = 0; j < k; ++j) off += (int)B.binom[B.L * kBinomStride + j];
        const uint16_t *lw = B.lowword + off;
        double sh = -shift;
        for (uint64_t m = h; m; m &= m - 1) sh += sw[B.L + __ffsll((long long)m) - 1];
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            double s = sh;
            for (uint32_t m = lw[r]; m; m &= m - 1) s += sw[__ffs(m) - 1];
            if (B.kept_map) {                   // truncated space: kept states only
                const int32_t m = B.kept_map[base + r];
                if (m >= 0) v[m] = (T)exp(s);
            } else {
                v[base + r] = (T)exp(s);
            }
        }
    }
}

// The same vector as a product of two factors, exp(sum over the state's high
// orbits - shift) * exp(sum over its low orbits): the low factor of every L-bit
// low word is tabulated once (elow, in the order of the lowword table), the
// high factor once per block, so a state costs one multiply instead of an
// FP64 exponential (GB300 executes FP64 at a small fraction of its FP32 rate).
__global__ void __launch_bounds__(256)
low_factor_kernel(const Blocks B, const OrbitWeights w, double *__restrict__ elow)
{
    const int nw = 1 << B.L;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nw; t += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (uint32_t m = B.lowword[t]; m; m &= m - 1) s += w.w[__ffs(m) - 1];
        elow[t] = exp(s);
    }
}

template <typename T>
__global__ void __launch_bounds__(256)
product_factored_kernel(const Blocks B, const OrbitWeights w, double shift, const double *__restrict__ elow,
                        T *__restrict__ v)
{
    __shared__ double s_high;
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b], base = B.blk_base[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        int off = 0;
        for (int j = 0; j < k; ++j) off += (int)B.binom[B.L * kBinomStride + j];
        __syncthreads();                          // s_high of the previous block is consumed
        if (threadIdx.x == 0) {
            double sh = -shift;
            for (uint64_t m = h; m; m &= m - 1) sh += w.w[B.L + __ffsll((long long)m) - 1];
            s_high = exp(sh);
        }
        __syncthreads();
        const double eh = s_high;
        const double *el = elow + off;
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            const T x = (T)(eh * el[r]);
            if (B.kept_map) {                     // truncated space: kept states only
                const int32_t m = B.kept_map[base + r];
                if (m >= 0) v[m] = x;
            } else {
                v[base + r] = x;
            }
        }
    }
}

// per CTA: M[i][j] += psi^2 n_i n_j, b[i] += psi^2 n_i log|psi| (shared accumulators)
__global__ void __launch_bounds__(256)
fit_kernel(const Blocks B, const double *__restrict__ v, double *__restrict__ part)
{
    extern __shared__ double acc[];              // omega*omega + omega
    const int om = B.omega, nacc = om * om + om;
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) acc[i] = 0.0;
    __syncthreads();
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b], base = B.blk_base[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        int off = 0;
        for (int j = 0; j < k; ++j) off += (int)B.binom[B.L * kBinomStride + j];
        const uint16_t *lw = B.lowword + off;
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            const double x = v[base + r];
            const double w2 = x * x;
            if (!(w2 > 1e-300)) continue;
            const double lg = log(fabs(x));
            const uint64_t s = (h << B.L) | (uint64_t)lw[r];
            for (uint64_t mi = s; mi; mi &= mi - 1) {
                const int i = __ffsll((long long)mi) - 1;
                atomicAdd(&acc[om * om + i], w2 * lg);
                for (uint64_t mj = s; mj; mj &= mj - 1) atomicAdd(&acc[i * om + __ffsll((long long)mj) - 1], w2);
            }
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nacc; i += blockDim.x) part[(size_t)blockIdx.x * nacc + i] = acc[i];
}

__global__ void fit_sum_kernel(const double *__restrict__ part, int nparts, int nacc, double *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nacc; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * nacc + i];
        out[i] = s;
    }
}

// batched product start: v[s] = exp(sum_{p in s} w[woff + p] - shift[problem])
template <typename T>
__global__ void __launch_bounds__(256)
batch_product_start_kernel(const BatchBlocks BB, const double *__restrict__ w, const int *__restrict__ woff,
                           const double *__restrict__ shift, T *__restrict__ v)
{
    for (long long b = blockIdx.x; b < BB.nblocks; b += gridDim.x) {
        const int pr = (int)BB.blk_prob[b];
        const BatchDesc dsc = BB.desc[pr];
        const double *wp = w + woff[pr];
        const uint64_t h = BB.blk_h[b], base = BB.blk_base[b];
        const int L = dsc.L;
        const int k = dsc.n - __popcll(h);
        const int nk = (int)BB.binom[L * kBinomStride + k];
        int off = 0;
        for (int j = 0; j < k; ++j) off += (int)BB.binom[L * kBinomStride + j];
        const uint16_t *lw = BB.lowword_all + dsc.tab_off + off;
        double sh = -shift[pr];
        for (uint64_t m = h; m; m &= m - 1) sh += wp[L + __ffsll((long long)m) - 1];
        T *vp = v + dsc.vec_off + base;
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            double sum = sh;
            for (uint32_t m = lw[r]; m; m &= m - 1) sum += wp[__ffs(m) - 1];
            vp[r] = (T)exp(sum);
        }
    }
}

}  // namespace

namespace pd {

// Batched warm start: one network pass over the orbits of all problems, then the
// product start vectors of every problem (storage dtype) into v (device).
int batch_mlp_start(struct ::pairdiag_mlp *m, const BatchBlocks &BB, int count, const int *omega, const int *n_pairs,
                    const double *e_all, const double *G_all, int dtype, void *v, cudaStream_t st)
{
    std::vector<int> woff(count);
    int rows = 0;
    for (int p = 0; p < count; ++p) { woff[p] = rows; rows += omega[p]; }
    std::vector<float> X((size_t)rows * kF);
    int64_t eo = 0, go = 0;
    for (int p = 0; p < count; ++p) {
        mlp_features(omega[p], n_pairs[p], e_all + eo, G_all + go, X.data() + (size_t)woff[p] * kF);
        eo += omega[p];
        go += (int64_t)omega[p] * omega[p];
    }
    PD_TRY(mlp_load_inputs(m, rows, X.data(), nullptr));
    PD_TRY(mlp_forward(m, rows));
    std::vector<float> o(rows);
    PD_CUDA(cudaMemcpyAsync(o.data(), m->out, sizeof(float) * rows, cudaMemcpyDeviceToHost, m->st));
    PD_CUDA(cudaStreamSynchronize(m->st));
    PD_TRY(check_tc(m));
    std::vector<double> w(o.begin(), o.end()), shift(count);
    for (int p = 0; p < count; ++p) {
        std::vector<double> srt(w.begin() + woff[p], w.begin() + woff[p] + omega[p]);
        std::sort(srt.begin(), srt.end(), std::greater<double>());
        double sh = 0.0;
        for (int i = 0; i < n_pairs[p]; ++i) sh += srt[i];
        shift[p] = sh;
    }
    double *dw = nullptr, *dsh = nullptr;
    int *dwo = nullptr;
    PD_CUDA(cudaMalloc(&dw, sizeof(double) * rows));
    cudaError_t e = cudaMalloc(&dsh, sizeof(double) * count);
    if (e == cudaSuccess) e = cudaMalloc(&dwo, sizeof(int) * count);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dw, w.data(), sizeof(double) * rows, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dsh, shift.data(), sizeof(double) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dwo, woff.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(BB.nblocks, sm_count() * 8));
        if (dtype == 0) batch_product_start_kernel<double><<<grid, 256, 0, st>>>(BB, dw, dwo, dsh, (double *)v);
        else batch_product_start_kernel<float><<<grid, 256, 0, st>>>(BB, dw, dwo, dsh, (float *)v);
        count_launches(1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(dw);
    if (dsh) cudaFree(dsh);
    if (dwo) cudaFree(dwo);
    PD_CUDA(e);
    return PD_OK;
}

// Per-orbit features of a problem (host): the Fermi level lam between the N-th
// and (N+1)-th lowest d_p = 2 e_p + G_pp, the pairing scale g = mean |G_ij|
// (i != j), the spread of d.
void mlp_features(int omega, int n, const double *e, const double *G, float *X)
{
    std::vector<double> d(omega);
    for (int p = 0; p < omega; ++p) d[p] = 2.0 * e[p] + G[p * omega + p];
    std::vector<int> order(omega);
    for (int p = 0; p < omega; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return d[a] < d[b]; });
    std::vector<int> rank(omega);
    for (int r = 0; r < omega; ++r) rank[order[r]] = r;
    const double lo = n > 0 ? d[order[n - 1]] : d[order[0]] - 1.0;
    const double hi = n < omega ? d[order[n]] : d[order[omega - 1]] + 1.0;
    const double lam = 0.5 * (lo + hi);
    double g = 0.0, mean = 0.0, var = 0.0;
    for (int i = 0; i < omega; ++i)
        for (int j = 0; j < omega; ++j)
            if (i != j) g += std::fabs(G[i * omega + j]);
    g = omega > 1 ? g / (omega * (omega - 1.0)) : 1.0;
    if (!(g > 0.0)) g = 1.0;
    for (int p = 0; p < omega; ++p) mean += d[p];
    mean /= omega;
    for (int p = 0; p < omega; ++p) var += (d[p] - mean) * (d[p] - mean);
    const double sd = std::sqrt(var / omega) + 1e-12;
    for (int p = 0; p < omega; ++p) {
        double row = 0.0;
        for (int j = 0; j < omega; ++j)
            if (j != p) row += G[p * omega + j];
        row = omega > 1 ? row / (omega - 1.0) : 0.0;
        float *x = X + (size_t)p * kF;
        const double u = (d[p] - lam) / g;
        x[0] = (float)(u / 10.0);
        x[1] = (float)std::tanh(u / omega);
        x[2] = rank[p] < n ? 1.0f : 0.0f;
        x[3] = (float)(G[p * omega + p] / g);
        x[4] = (float)(row / g);
        x[5] = (float)((double)n / omega);
        x[6] = (float)(omega / 32.0);
        x[7] = (float)((rank[p] - n + 0.5) / omega);
        x[8] = (float)((d[p] - lam) / sd);
        x[9] = (float)(g / sd);
        x[10] = (float)std::tanh(u);
        x[11] = (float)std::tanh(u / 4.0);
        for (int f = 12; f < kF; ++f) x[f] = 0.0f;
    }
}

// weights w (host, [omega]) -> start vector (device) of storage dtype.
// scratch: 2^L device doubles for the low-word factors (nullable: then one
// FP64 exponential per state).  Asynchronous on st.
int product_start(const Blocks &B, const double *w_host, int dtype, void *v, cudaStream_t st, double *scratch)
{
    std::vector<double> w(w_host, w_host + B.omega);
    std::vector<double> srt(w);
    std::sort(srt.begin(), srt.end(), std::greater<double>());
    double shift = 0.0;
    for (int i = 0; i < B.n; ++i) shift += srt[i];        // the largest exponent over the basis
    OrbitWeights ow{};
    for (int p = 0; p < B.omega; ++p) ow.w[p] = w[p];
    // the factors stay finite when neither partial exponent can pass 700
    double lo_abs = 0.0, hi_abs = std::fabs(shift);
    for (int p = 0; p < B.omega; ++p) (p < B.L ? lo_abs : hi_abs) += std::fabs(w[p]);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(B.nblocks, sm_count() * 4));
    if (scratch && lo_abs < 700.0 && hi_abs < 700.0) {
        const int tgrid = ((1 << B.L) + 255) / 256;
        low_factor_kernel<<<tgrid, 256, 0, st>>>(B, ow, scratch);
        if (dtype == 0) product_factored_kernel<double><<<grid, 256, 0, st>>>(B, ow, shift, scratch, (double *)v);
        else product_factored_kernel<float><<<grid, 256, 0, st>>>(B, ow, shift, scratch, (float *)v);
        count_launches(2);
    } else {
        if (dtype == 0) product_start_kernel<double><<<grid, 256, 0, st>>>(B, ow, shift, (double *)v);
        else product_start_kernel<float><<<grid, 256, 0, st>>>(B, ow, shift, (float *)v);
        count_launches(1);
    }
    PD_CUDA(cudaGetLastError());
    return PD_OK;
}

// least-squares per-orbit weights of a normalised FP64 vector v (device)
int product_fit(const Blocks &B, const double *v, double *w_out, cudaStream_t st)
{
    const int om = B.omega, nacc = om * om + om;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(B.nblocks, sm_count() * 2));
    double *part = nullptr, *sum = nullptr;
    PD_CUDA(cudaMalloc(&part, sizeof(double) * (size_t)grid * nacc));
    cudaError_t e = cudaMalloc(&sum, sizeof(double) * nacc);
    std::vector<double> h(nacc);
    if (e == cudaSuccess) {
        const size_t smem = sizeof(double) * nacc;
        cudaFuncSetAttribute(fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fit_kernel<<<grid, 256, smem, st>>>(B, v, part);
        fit_sum_kernel<<<(nacc + 255) / 256, 256, 0, st>>>(part, grid, nacc, sum);
        count_launches(2);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), sum, sizeof(double) * nacc, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    cudaFree(part);
    if (sum) cudaFree(sum);
    PD_CUDA(e);
    // solve (M + eps I) w = b by Gaussian elimination with partial pivoting
    std::vector<double> M(h.begin(), h.begin() + om * om), b(h.begin() + om * om, h.end());
    double tr = 0.0;
    for (int i = 0; i < om; ++i) tr += M[i * om + i];
    for (int i = 0; i < om; ++i) M[i * om + i] += 1e-9 * (tr / om + 1e-300);   // ridge: orbits that are
                                                                                // (almost) always full or empty
    for (int c = 0; c < om; ++c) {
        int piv = c;
        for (int r = c + 1; r < om; ++r)
            if (std::fabs(M[r * om + c]) > std::fabs(M[piv * om + c])) piv = r;
        if (piv != c) {
            for (int j = 0; j < om; ++j) std::swap(M[c * om + j], M[piv * om + j]);
            std::swap(b[c], b[piv]);
        }
        const double dv = M[c * om + c];
        if (dv == 0.0) return fail(PD_ECUDA, "product fit: singular normal equations");
        for (int r = c + 1; r < om; ++r) {
            const double f = M[r * om + c] / dv;
            if (f == 0.0) continue;
            for (int j = c; j < om; ++j) M[r * om + j] -= f * M[c * om + j];
            b[r] -= f * b[c];
        }
    }
    for (int c = om - 1; c >= 0; --c) {
        double s = b[c];
        for (int j = c + 1; j < om; ++j) s -= M[c * om + j] * w_out[j];
        w_out[c] = s / M[c * om + c];
    }
    double mean = 0.0;                               // remove the free constant (a global scale)
    for (int i = 0; i < om; ++i) mean += w_out[i];
    mean /= om;
    for (int i = 0; i < om; ++i) w_out[i] -= mean;
    return PD_OK;
}

int mlp_predict(pairdiag_mlp *m, int omega, int n, const double *e, const double *G, double *w_out)
{
    std::vector<float> X((size_t)omega * kF);
    mlp_features(omega, n, e, G, X.data());
    PD_TRY(mlp_load_inputs(m, omega, X.data(), nullptr));
    PD_TRY(mlp_forward(m, omega));
    std::vector<float> o(omega);
    PD_CUDA(cudaMemcpyAsync(o.data(), m->out, sizeof(float) * omega, cudaMemcpyDeviceToHost, m->st));
    PD_CUDA(cudaStreamSynchronize(m->st));
    PD_TRY(check_tc(m));
    for (int i = 0; i < omega; ++i) w_out[i] = o[i];
    return PD_OK;
}

}  // namespace pd

extern "C" {

int pairdiag_mlp_create(uint64_t seed, pairdiag_mlp_t **out)
{
    if (!out) return fail(PD_EINVAL, "null argument");
    *out = nullptr;
    pairdiag_mlp *m = new pairdiag_mlp();
    // He-style initialisation from a counter-based generator
    std::vector<float> th(kNParams, 0.0f);
    auto uni = [&](uint64_t i) {
        uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
    };
    auto fill = [&](int off, int n, double scale) {
        for (int i = 0; i < n; ++i) th[off + i] = (float)(scale * uni((uint64_t)(off + i)));
    };
    fill(oW1, kF * kH, std::sqrt(6.0 / kF));
    fill(oW2, kH * kH, std::sqrt(6.0 / kH));
    fill(oW3, kH * kH, std::sqrt(6.0 / kH));
    fill(ow4, kH, std::sqrt(3.0 / kH));
    int st = PD_OK;
    do {
        if (cudaMalloc(&m->theta, sizeof(float) * kNParams) != cudaSuccess ||
            cudaMalloc(&m->wb, sizeof(bf16) * kNParams) != cudaSuccess ||
            cudaMalloc(&m->grad, sizeof(float) * kNParams) != cudaSuccess ||
            cudaMalloc(&m->m1, sizeof(float) * kNParams) != cudaSuccess ||
            cudaMalloc(&m->m2, sizeof(float) * kNParams) != cudaSuccess ||
            cudaMalloc(&m->loss, sizeof(double)) != cudaSuccess || cudaMalloc(&m->err, sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            st = fail(PD_ENOMEM, "mlp: allocation failed");
            break;
        }
        if (cudaMemcpy(m->theta, th.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemset(m->m1, 0, sizeof(float) * kNParams) != cudaSuccess ||
            cudaMemset(m->m2, 0, sizeof(float) * kNParams) != cudaSuccess ||
            cudaMemset(m->err, 0, sizeof(int)) != cudaSuccess)
            st = fail(PD_ECUDA, "mlp: initialisation failed");
    } while (0);
    if (st != PD_OK) {
        pairdiag_mlp_destroy(m);
        return st;
    }
    *out = m;
    return PD_OK;
}

void pairdiag_mlp_destroy(pairdiag_mlp_t *m)
{
    if (!m) return;
    cudaStreamSynchronize(m->st);
    mlp_free_work(m);
    void *p[] = {m->theta, m->wb, m->grad, m->m1, m->m2, m->loss, m->err};
    for (void *q : p)
        if (q) cudaFree(q);
    delete m;
}

int pairdiag_mlp_num_params(void) { return kNParams; }

int pairdiag_mlp_get_params(const pairdiag_mlp_t *m, float *out)
{
    if (!m || !out) return fail(PD_EINVAL, "null argument");
    PD_CUDA(cudaMemcpy(out, m->theta, sizeof(float) * kNParams, cudaMemcpyDeviceToHost));
    return PD_OK;
}

int pairdiag_mlp_set_params(pairdiag_mlp_t *m, const float *in)
{
    if (!m || !in) return fail(PD_EINVAL, "null argument");
    PD_CUDA(cudaMemcpy(m->theta, in, sizeof(float) * kNParams, cudaMemcpyHostToDevice));
    PD_CUDA(cudaMemset(m->m1, 0, sizeof(float) * kNParams));
    PD_CUDA(cudaMemset(m->m2, 0, sizeof(float) * kNParams));
    m->steps = 0;
    return PD_OK;
}

int pairdiag_mlp_features(int omega, int n_pairs, const double *e, const double *G, float *X)
{
    if (omega < 1 || omega > kMaxOmega || n_pairs < 0 || n_pairs > omega || !e || !G || !X)
        return fail(PD_EINVAL, "bad argument");
    mlp_features(omega, n_pairs, e, G, X);
    return PD_OK;
}

int pairdiag_mlp_forward(pairdiag_mlp_t *m, int rows, const float *X, float *out)
{
    if (!m || rows < 1 || !X || !out) return fail(PD_EINVAL, "bad argument");
    PD_TRY(mlp_load_inputs(m, rows, X, nullptr));
    PD_TRY(mlp_forward(m, rows));
    PD_CUDA(cudaMemcpyAsync(out, m->out, sizeof(float) * rows, cudaMemcpyDeviceToHost, m->st));
    PD_CUDA(cudaStreamSynchronize(m->st));
    return check_tc(m);
}

int pairdiag_mlp_loss_grad(pairdiag_mlp_t *m, int rows, const float *X, const float *target, double *loss,
                           float *grad)
{
    if (!m || rows < 1 || !X || !target || !loss || !grad) return fail(PD_EINVAL, "bad argument");
    PD_TRY(mlp_load_inputs(m, rows, X, target));
    PD_TRY(mlp_forward(m, rows));
    PD_TRY(mlp_backward(m, rows));
    PD_CUDA(cudaMemcpyAsync(grad, m->grad, sizeof(float) * kNParams, cudaMemcpyDeviceToHost, m->st));
    PD_CUDA(cudaMemcpyAsync(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost, m->st));
    PD_CUDA(cudaStreamSynchronize(m->st));
    return check_tc(m);
}

int pairdiag_mlp_train(pairdiag_mlp_t *m, int rows, const float *X, const float *target, int steps, double lr,
                       double *loss_history)
{
    if (!m || rows < 1 || !X || !target || steps < 0 || !(lr > 0.0)) return fail(PD_EINVAL, "bad argument");
    PD_TRY(mlp_load_inputs(m, rows, X, target));
    const float b1 = 0.9f, b2 = 0.999f;
    std::vector<double> hist(steps);
    double *d_hist = nullptr;
    if (loss_history && steps > 0) PD_CUDA(cudaMalloc(&d_hist, sizeof(double) * steps));
    int rc = PD_OK;
    for (int s = 0; s < steps && rc == PD_OK; ++s) {
        rc = mlp_forward(m, rows);
        if (rc == PD_OK) rc = mlp_backward(m, rows);
        if (rc != PD_OK) break;
        ++m->steps;
        const float c1 = 1.0f - std::pow(b1, (float)m->steps), c2 = 1.0f - std::pow(b2, (float)m->steps);
        adam_kernel<<<grid1(kNParams), 256, 0, m->st>>>(m->theta, m->grad, m->m1, m->m2, kNParams, (float)lr, b1, b2,
                                                        c1, c2, 1e-8f);
        count_launches(1);
        if (d_hist) cudaMemcpyAsync(d_hist + s, m->loss, sizeof(double), cudaMemcpyDeviceToDevice, m->st);
    }
    if (rc == PD_OK && d_hist) {
        cudaMemcpyAsync(loss_history, d_hist, sizeof(double) * steps, cudaMemcpyDeviceToHost, m->st);
    }
    const cudaError_t e = cudaStreamSynchronize(m->st);
    if (d_hist) cudaFree(d_hist);
    if (rc != PD_OK) return rc;
    PD_CUDA(e);
    return check_tc(m);
}

int pairdiag_mlp_buffer(const pairdiag_mlp_t *m, int which, int rows, float *out)
{
    if (!m || !out || rows < 1) return fail(PD_EINVAL, "bad argument");
    if (rows > m->cap) return fail(PD_EINVAL, "rows=%d beyond the last pass (%d rows)", rows, m->cap);
    const size_t nh = (size_t)rows * kH;
    const float *f = nullptr;
    const bf16 *b = nullptr;
    size_t n = nh;
    switch (which) {
    case PD_MLP_Z1: f = m->Z1; break;
    case PD_MLP_A1: b = m->A1; break;
    case PD_MLP_Z2: f = m->Z2; break;
    case PD_MLP_A2: b = m->A2; break;
    case PD_MLP_Z3: f = m->Z3; break;
    case PD_MLP_A3: b = m->A3; break;
    case PD_MLP_OUT: f = m->out; n = (size_t)rows; break;
    case PD_MLP_DOUT: f = m->dout; n = (size_t)rows; break;
    case PD_MLP_DZ3: b = m->dZ3; break;
    case PD_MLP_DA2: f = m->dA2; break;
    case PD_MLP_DZ2: b = m->dZ2; break;
    case PD_MLP_DA1: f = m->dA1; break;
    case PD_MLP_DZ1: b = m->dZ1; break;
    default: return fail(PD_EINVAL, "unknown buffer %d", which);
    }
    PD_CUDA(cudaStreamSynchronize(m->st));
    if (f) {
        PD_CUDA(cudaMemcpy(out, f, sizeof(float) * n, cudaMemcpyDeviceToHost));
    } else {
        std::vector<bf16> tmp(n);
        PD_CUDA(cudaMemcpy(tmp.data(), b, sizeof(bf16) * n, cudaMemcpyDeviceToHost));
        for (size_t i = 0; i < n; ++i) out[i] = __bfloat162float(tmp[i]);
    }
    return PD_OK;
}

}  // extern "C"
