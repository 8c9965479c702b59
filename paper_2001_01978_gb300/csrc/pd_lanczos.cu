// pd_lanczos.cu -- the vector algebra of restarted Lanczos (Algorithm 2 with
// full Gram-Schmidt reorthogonalisation and restart, Sec. 3.4) and the small
// symmetric tridiagonal eigenproblem of its L matrix.
//
// Streaming kernels run on a fixed persistent grid; each CTA writes partial
// sums to a scratch array and a one-CTA kernel adds them in a fixed order, so
// every reduction is deterministic.  Products are formed in FP64 whatever the
// storage type (an FP32 x FP32 product is exact in FP64).
#include "pd_internal.h"

#include <cfloat>
#include <cmath>

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;             // vectors handled per pass of a multi-dot
constexpr int kGrid = 152 * 4;

__device__ __forceinline__ double ld(const double *p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ double ld(const float *p, int64_t i) { return (double)__ldg(p + i); }

// block-wide sum of one double per thread; result valid in thread 0
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// partial[b*kMaxWindow + j] = sum over this CTA's elements of Q_j[i] p[i]
template <typename T>
__global__ void __launch_bounds__(kThreads)
multidot_kernel(const T *__restrict__ Q, int64_t ldq, int m, const T *__restrict__ p, int64_t n,
                double *__restrict__ part, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ double sh[kThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int j0 = 0; j0 < m; j0 += kGroup) {
        double acc[kGroup];
#pragma unroll
        for (int u = 0; u < kGroup; ++u) acc[u] = 0.0;
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
            const double pv = ld(p, i);
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m) acc[u] += ld(Q, (int64_t)(j0 + u) * ldq + i) * pv;
        }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
            if (j0 + u < m) {
                const double s = block_sum(acc[u], sh);
                if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow + j0 + u] = s;
            }
        }
    }
}

// Float-float accumulation of exact products with FP32 instructions only:
// a*b = p + pe exactly (FMA), and (hi, lo) += p + pe with Knuth's TwoSum.  This
// gives close to FP64 accuracy for dot products of FP32 vectors without FP64
// arithmetic, which GB300 executes at a small fraction of its FP32 rate.
__device__ __forceinline__ void ff_add_prod(float &hi, float &lo, float a, float b)
{
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float t = hi + p;
    const float z = t - hi;
    const float e = (hi - (t - z)) + (p - z);
    hi = t;
    lo += e + pe;
}

// multi-dot of FP32 vectors, float-float per thread, FP64 across threads
__global__ void __launch_bounds__(kThreads)
multidot_f32_kernel(const float *__restrict__ Q, int64_t ldq, int m, const float *__restrict__ p, int64_t n,
                    double *__restrict__ part, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ double sh[kThreads / 32];
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int j0 = 0; j0 < m; j0 += kGroup) {
        float hi[kGroup], lo[kGroup];
#pragma unroll
        for (int u = 0; u < kGroup; ++u) hi[u] = lo[u] = 0.0f;
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
            const float pv = __ldg(p + i);
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m) ff_add_prod(hi[u], lo[u], __ldg(Q + (int64_t)(j0 + u) * ldq + i), pv);
        }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
            if (j0 + u < m) {
                const double s = block_sum((double)hi[u] + (double)lo[u], sh);
                if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow + j0 + u] = s;
            }
        }
    }
}

// Lanczos recurrence fused with the projections of one Gram-Schmidt pass:
//   p <- p - alpha q_i - beta_{i-1} q_{i-1}   (Algorithm 2; alpha = S->c1[0])
//   part <- per-CTA partial sums of Q_j^T p for j <= i (after the update)
// Elements are visited in the same order by the same thread in every group, so
// the groups after the first read back this thread's own updated values.
template <typename T>
__global__ void __launch_bounds__(kThreads)
recur_project_kernel(const T *__restrict__ Q, int64_t ldq, int i, const LanczosScalars *__restrict__ S,
                     T *__restrict__ p, int64_t n, double *__restrict__ part, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ double sh[kThreads / 32];
    const int m = i + 1;
    const T a = (T)S->c1[0];
    const T b = (T)(i > 0 ? S->beta[i - 1] : 0.0);
    const T *qi = Q + (int64_t)i * ldq;
    const T *qm = Q + (int64_t)(i > 0 ? i - 1 : 0) * ldq;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int j0 = 0; j0 < m; j0 += kGroup) {
        float hi[kGroup], lo[kGroup];     // used by the FP32 path
        double acc[kGroup];               // used by the FP64 path
#pragma unroll
        for (int u = 0; u < kGroup; ++u) { hi[u] = lo[u] = 0.0f; acc[u] = 0.0; }
        for (int64_t e = blockIdx.x * (int64_t)kThreads + threadIdx.x; e < n; e += stride) {
            T v;
            if (j0 == 0) {
                v = p[e];
                if constexpr (sizeof(T) == 4) {
                    v = fmaf(-a, __ldg(qi + e), v);
                    if (i > 0) v = fmaf(-b, __ldg(qm + e), v);
                } else {
                    v = fma(-a, __ldg(qi + e), v);
                    if (i > 0) v = fma(-b, __ldg(qm + e), v);
                }
                p[e] = v;
            } else {
                v = p[e];
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u) {
                if (j0 + u < m) {
                    const T q = __ldg(Q + (int64_t)(j0 + u) * ldq + e);
                    if constexpr (sizeof(T) == 4) ff_add_prod(hi[u], lo[u], q, v);
                    else acc[u] = fma((double)q, (double)v, acc[u]);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
            if (j0 + u < m) {
                const double val = (sizeof(T) == 4) ? (double)hi[u] + (double)lo[u] : acc[u];
                const double s = block_sum(val, sh);
                if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow + j0 + u] = s;
            }
        }
    }
}

// out[j] = sum_b part[b*kMaxWindow + j]: one warp per output, each lane a fixed
// strided subset, then a fixed xor-shuffle tree (deterministic)
__global__ void reduce_kernel(const double *__restrict__ part, int nb, int m, double *__restrict__ out,
                              const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (j >= m) return;
    double s = 0.0;
#pragma unroll 4
    for (int b = lane; b < nb; b += 32) s += part[b * kMaxWindow + j];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[j] = s;
}

inline void reduce(const double *part, int nb, int m, double *out, cudaStream_t st, const int *skip = nullptr)
{
    reduce_kernel<<<(m + 7) / 8, 256, 0, st>>>(part, nb, m, out, skip);
}

// p -= sum_j c_j Q_j ; optional ||p||^2 partials (of the stored, rounded values)
template <typename T>
__global__ void __launch_bounds__(kThreads)
update_kernel(const T *__restrict__ Q, int64_t ldq, int m, const double *__restrict__ c,
              T *__restrict__ p, int64_t n, double *__restrict__ part, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ double sc[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < m; j += kThreads) sc[j] = c[j];
    __syncthreads();
    double nrm = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
        double v = (double)p[i];
        for (int j = 0; j < m; ++j) v -= sc[j] * ld(Q, (int64_t)j * ldq + i);
        const T t = (T)v;
        p[i] = t;
        nrm += (double)t * (double)t;
    }
    if (part) {
        const double s = block_sum(nrm, sh);
        if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = s;
    }
}

// p -= sum_j c_j Q_j with FP32 FMAs (the result is stored in FP32 anyway; the
// second Gram-Schmidt pass removes what this rounding leaves along Q)
__global__ void __launch_bounds__(kThreads)
update_f32_kernel(const float *__restrict__ Q, int64_t ldq, int m, const double *__restrict__ c,
                  float *__restrict__ p, int64_t n, double *__restrict__ part, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ float sc[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < m; j += kThreads) sc[j] = (float)c[j];
    __syncthreads();
    float hi = 0.0f, lo = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
        float v = p[i];
        for (int j = 0; j < m; ++j) v = fmaf(-sc[j], __ldg(Q + (int64_t)j * ldq + i), v);
        p[i] = v;
        ff_add_prod(hi, lo, v, v);
    }
    if (part) {
        const double s = block_sum((double)hi + (double)lo, sh);
        if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = s;
    }
}

__global__ void scale_f32_kernel(const float *__restrict__ src, float *__restrict__ dst, int64_t n,
                                 const double *__restrict__ div, int is_norm2, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const double d = is_norm2 ? sqrt(*div) : *div;
    const float f = (d > 0.0) ? (float)(1.0 / d) : 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = src[i] * f;
}

template <typename T>
__global__ void scale_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t n,
                             const double *__restrict__ div, int is_norm2, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const double d = is_norm2 ? sqrt(*div) : *div;
    const double f = (d > 0.0) ? 1.0 / d : 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (T)((double)src[i] * f);
}

__global__ void finalize_kernel(LanczosScalars *S, int i)
{
    if (threadIdx.x != 0 || blockIdx.x != 0 || S->broken) return;
    const double a = S->c1[0] + S->c2[i];
    const double b = sqrt(S->norm2);
    S->alpha[i] = a;
    S->beta[i] = b;
    const double row = fabs(a) + b + (i > 0 ? S->beta[i - 1] : 0.0);
    const double tn = fmax(S->tnorm, row);
    S->tnorm = tn;
    S->used = i + 1;
    if (!(b > 1e-13 * tn)) S->broken = 1;        // invariant subspace found (or a NaN)
}

__global__ void cycle_reset_kernel(LanczosScalars *S)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    S->used = 0;
    S->broken = 0;
    S->tnorm = 0.0;
}

// ---- symmetric tridiagonal eigenproblem (one warp) --------------------------
// Number of eigenvalues below x (Sturm sequence of the LDL^T pivots of T - xI).
__device__ int sturm_count(const double *a, const double *b2, int m, double x, double tiny)
{
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
        d = a[i] - x - (i > 0 ? b2[i - 1] / d : 0.0);
        if (d == 0.0) d = -tiny;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// j-th smallest eigenvalue (j = 1, 2, ...) by 33-way multisection across the warp
__device__ double kth_eigenvalue(const double *a, const double *b2, int m, int j, double lo, double hi,
                                 double tiny)
{
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < 64; ++it) {
        const double w = hi - lo;
        if (w <= 2.0 * DBL_EPSILON * fmax(fabs(lo), fabs(hi)) || w <= tiny) break;
        const double xl = lo + w * (double)(lane + 1) / 33.0;
        const int c = sturm_count(a, b2, m, xl, tiny);
        const unsigned below = __ballot_sync(0xffffffffu, c < j);    // eigenvalue j lies above xl
        const int nb = __popc(below);                                 // the points below are a prefix
        const double new_lo = nb > 0 ? __shfl_sync(0xffffffffu, xl, nb - 1) : lo;
        const double new_hi = nb < 32 ? __shfl_sync(0xffffffffu, xl, nb < 32 ? nb : 31) : hi;
        if (new_lo == lo && new_hi == hi) break;
        lo = new_lo;
        hi = new_hi;
    }
    return 0.5 * (lo + hi);
}

// Solve (T - theta I) z = r for a symmetric tridiagonal T by Gaussian
// elimination with partial pivoting (row i and i+1 may swap; the upper factor
// then has two superdiagonals).  Zero pivots are replaced by `tiny`.
__device__ void tridiag_solve(const double *a, const double *b, int m, double theta, double *r,
                              double *u0, double *u1, double *u2, double tiny)
{
    // current row i: (c0, c1, c2) in columns i, i+1, i+2
    double c0 = a[0] - theta, c1 = (m > 1 ? b[0] : 0.0), c2 = 0.0;
    for (int i = 0; i < m - 1; ++i) {
        // next row i+1: columns i, i+1, i+2
        double n0 = b[i], n1 = a[i + 1] - theta, n2 = (i + 2 < m ? b[i + 1] : 0.0);
        if (fabs(n0) > fabs(c0)) {      // swap rows i and i+1
            double t;
            t = c0; c0 = n0; n0 = t;
            t = c1; c1 = n1; n1 = t;
            t = c2; c2 = n2; n2 = t;
            t = r[i]; r[i] = r[i + 1]; r[i + 1] = t;
        }
        if (c0 == 0.0) c0 = tiny;
        const double mu = n0 / c0;
        u0[i] = c0; u1[i] = c1; u2[i] = c2;
        r[i + 1] -= mu * r[i];
        c0 = n1 - mu * c1;
        c1 = n2 - mu * c2;
        c2 = 0.0;
    }
    if (c0 == 0.0) c0 = tiny;
    u0[m - 1] = c0; u1[m - 1] = 0.0; u2[m - 1] = 0.0;
    for (int i = m - 1; i >= 0; --i) {
        double s = r[i];
        if (i + 1 < m) s -= u1[i] * r[i + 1];
        if (i + 2 < m) s -= u2[i] * r[i + 2];
        r[i] = s / u0[i];
    }
}

__global__ void tridiag_kernel(LanczosScalars *S, int m)
{
    __shared__ double a[kMaxWindow], b[kMaxWindow], b2[kMaxWindow];
    __shared__ double z[kMaxWindow], u0[kMaxWindow], u1[kMaxWindow], u2[kMaxWindow];
    const int lane = threadIdx.x;
    if (m <= 0) m = S->used;
    if (m < 1 || m > kMaxWindow) return;
    for (int i = lane; i < m; i += 32) {
        a[i] = S->alpha[i];
        b[i] = (i + 1 < m) ? S->beta[i] : 0.0;
        b2[i] = b[i] * b[i];
    }
    __syncwarp();
    if (m == 1) {
        if (lane == 0) { S->theta[0] = a[0]; S->theta[1] = INFINITY; S->s[0] = 1.0; }
        return;
    }
    // Gershgorin interval and the scale of T
    double lo = INFINITY, hi = -INFINITY, scale = 0.0;
    for (int i = 0; i < m; ++i) {
        const double rad = fabs(b[i]) + (i > 0 ? fabs(b[i - 1]) : 0.0);
        lo = fmin(lo, a[i] - rad);
        hi = fmax(hi, a[i] + rad);
        scale = fmax(scale, fabs(a[i]) + rad);
    }
    const double tiny = fmax(scale, DBL_MIN) * DBL_EPSILON;
    lo -= tiny; hi += tiny;
    const double t1 = kth_eigenvalue(a, b2, m, 1, lo, hi, DBL_MIN);
    const double t2 = kth_eigenvalue(a, b2, m, 2, lo, hi, DBL_MIN);
    if (lane == 0) {
        // inverse iteration for the eigenvector of t1
        for (int i = 0; i < m; ++i) z[i] = 1.0;
        for (int it = 0; it < 3; ++it) {
            tridiag_solve(a, b, m, t1, z, u0, u1, u2, tiny);
            double nrm = 0.0;
            for (int i = 0; i < m; ++i) nrm += z[i] * z[i];
            nrm = sqrt(nrm);
            for (int i = 0; i < m; ++i) z[i] /= nrm;
        }
        double big = 0.0; int ib = 0;                 // fix the sign: largest component positive
        for (int i = 0; i < m; ++i) if (fabs(z[i]) > big) { big = fabs(z[i]); ib = i; }
        const double sg = z[ib] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < m; ++i) S->s[i] = sg * z[i];
        S->theta[0] = t1;
        S->theta[1] = t2;
    }
}

// Q0 <- sum_j s_j Q_j (in place; each element is read before it is written)
template <typename T>
__global__ void __launch_bounds__(kThreads)
ritz_kernel(T *__restrict__ Q, int64_t ldq, const int *__restrict__ m_dev, const double *__restrict__ s,
            int64_t n, double *__restrict__ part)
{
    const int m = *m_dev;
    __shared__ double ss[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < m; j += kThreads) ss[j] = s[j];
    __syncthreads();
    double nrm = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
        double v = 0.0;
        for (int j = 0; j < m; ++j) v += ss[j] * (double)Q[(int64_t)j * ldq + i];
        const T t = (T)v;
        Q[i] = t;
        nrm += (double)t * (double)t;
    }
    const double sum = block_sum(nrm, sh);
    if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = sum;
}

__global__ void __launch_bounds__(kThreads)
ritz_f32_kernel(float *__restrict__ Q, int64_t ldq, const int *__restrict__ m_dev, const double *__restrict__ s,
                int64_t n, double *__restrict__ part)
{
    const int m = *m_dev;
    __shared__ float ss[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < m; j += kThreads) ss[j] = (float)s[j];
    __syncthreads();
    float hi = 0.0f, lo = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
        float v = 0.0f;
        for (int j = 0; j < m; ++j) v = fmaf(ss[j], Q[(int64_t)j * ldq + i], v);
        Q[i] = v;
        ff_add_prod(hi, lo, v, v);
    }
    const double sum = block_sum((double)hi + (double)lo, sh);
    if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = sum;
}

// counter-based SplitMix64 (Steele, Lea & Flood 2014) -> uniform [-1, 1)
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i)
{
    uint64_t z = seed + (i + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

template <typename T>
__global__ void random_kernel(T *__restrict__ q, int64_t n, uint64_t seed)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        q[i] = (T)splitmix_uniform(seed, (uint64_t)i);
}

template <typename D, typename S>
__global__ void convert_kernel(D *__restrict__ dst, const S *__restrict__ src, int64_t n)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (D)src[i];
}

__global__ void __launch_bounds__(kThreads)
residual_kernel(const double *__restrict__ a, const double *__restrict__ b,
                const double *__restrict__ lambda, double *__restrict__ dst, int64_t n,
                double *__restrict__ part)
{
    __shared__ double sh[kThreads / 32];
    const double lam = *lambda;
    double nrm = 0.0;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += stride) {
        const double r = a[i] - lam * b[i];
        if (dst) dst[i] = r;
        nrm += r * r;
    }
    const double s = block_sum(nrm, sh);
    if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = s;
}

int grid_for(int64_t n)
{
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > kGrid) g = kGrid;
    return (int)(g > 0 ? g : 1);
}

}  // namespace

int vec_grid() { return kGrid; }

cudaError_t multidot_launch(int dtype, const void *Q, int64_t ld, int m, const void *p, int64_t n,
                            double *partials, double *out, cudaStream_t st, const int *skip)
{
    const int g = grid_for(n);
    if (dtype == 0)
        multidot_kernel<double><<<g, kThreads, 0, st>>>((const double *)Q, ld, m, (const double *)p, n, partials, skip);
    else
        multidot_f32_kernel<<<g, kThreads, 0, st>>>((const float *)Q, ld, m, (const float *)p, n, partials, skip);
    reduce(partials, g, m, out, st, skip);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t update_launch(int dtype, const void *Q, int64_t ld, int m, const double *c, void *p,
                          int64_t n, double *partials, double *norm_out, cudaStream_t st, const int *skip)
{
    const int g = grid_for(n);
    double *part = norm_out ? partials : nullptr;
    if (dtype == 0)
        update_kernel<double><<<g, kThreads, 0, st>>>((const double *)Q, ld, m, c, (double *)p, n, part, skip);
    else
        update_f32_kernel<<<g, kThreads, 0, st>>>((const float *)Q, ld, m, c, (float *)p, n, part, skip);
    if (norm_out) reduce(partials, g, 1, norm_out, st, skip);
    count_launches((norm_out ? 2 : 1));
    return cudaGetLastError();
}

cudaError_t scale_launch(int dtype, const void *src, void *dst, int64_t n, const double *div,
                         int div_is_norm2, cudaStream_t st, const int *skip)
{
    const int g = grid_for(n);
    if (dtype == 0)
        scale_kernel<double><<<g, kThreads, 0, st>>>((const double *)src, (double *)dst, n, div, div_is_norm2, skip);
    else
        scale_f32_kernel<<<g, kThreads, 0, st>>>((const float *)src, (float *)dst, n, div, div_is_norm2, skip);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t recur_project_launch(int dtype, const void *Q, int64_t ld, int i, const LanczosScalars *S,
                                 void *p, int64_t n, double *partials, double *out, cudaStream_t st,
                                 const int *skip)
{
    const int g = grid_for(n);
    if (dtype == 0)
        recur_project_kernel<double><<<g, kThreads, 0, st>>>((const double *)Q, ld, i, S, (double *)p, n, partials, skip);
    else
        recur_project_kernel<float><<<g, kThreads, 0, st>>>((const float *)Q, ld, i, S, (float *)p, n, partials, skip);
    reduce(partials, g, i + 1, out, st, skip);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t finalize_step_launch(LanczosScalars *S, int i, cudaStream_t st)
{
    finalize_kernel<<<1, 32, 0, st>>>(S, i);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t cycle_reset_launch(LanczosScalars *S, cudaStream_t st)
{
    cycle_reset_kernel<<<1, 32, 0, st>>>(S);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t tridiag_launch(LanczosScalars *S, int m, cudaStream_t st)
{
    tridiag_kernel<<<1, 32, 0, st>>>(S, m);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t ritz_launch(int dtype, void *Q, int64_t ld, const int *m_dev, const double *s, int64_t n,
                        double *partials, double *norm_out, cudaStream_t st)
{
    const int g = grid_for(n);
    if (dtype == 0)
        ritz_kernel<double><<<g, kThreads, 0, st>>>((double *)Q, ld, m_dev, s, n, partials);
    else
        ritz_f32_kernel<<<g, kThreads, 0, st>>>((float *)Q, ld, m_dev, s, n, partials);
    reduce(partials, g, 1, norm_out, st);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t random_start_launch(int dtype, void *q, int64_t n, uint64_t seed, cudaStream_t st)
{
    const int g = grid_for(n);
    if (dtype == 0) random_kernel<double><<<g, kThreads, 0, st>>>((double *)q, n, seed);
    else random_kernel<float><<<g, kThreads, 0, st>>>((float *)q, n, seed);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t convert_launch(int dst_dtype, void *dst, int src_dtype, const void *src, int64_t n,
                           cudaStream_t st)
{
    const int g = grid_for(n);
    if (dst_dtype == 0 && src_dtype == 1)
        convert_kernel<double, float><<<g, kThreads, 0, st>>>((double *)dst, (const float *)src, n);
    else if (dst_dtype == 1 && src_dtype == 0)
        convert_kernel<float, double><<<g, kThreads, 0, st>>>((float *)dst, (const double *)src, n);
    else if (dst_dtype == 0)
        convert_kernel<double, double><<<g, kThreads, 0, st>>>((double *)dst, (const double *)src, n);
    else
        convert_kernel<float, float><<<g, kThreads, 0, st>>>((float *)dst, (const float *)src, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t residual_launch(const double *a, const double *b, const double *lambda, double *dst,
                            int64_t n, double *partials, double *norm_out, cudaStream_t st)
{
    const int g = grid_for(n);
    residual_kernel<<<g, kThreads, 0, st>>>(a, b, lambda, dst, n, partials);
    reduce(partials, g, 1, norm_out, st);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace pd
