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
                double *__restrict__ part)
{
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

// out[j] = sum_b part[b*kMaxWindow + j], fixed order
__global__ void reduce_kernel(const double *__restrict__ part, int nb, int m, double *__restrict__ out)
{
    const int j = threadIdx.x;
    if (j >= m) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[b * kMaxWindow + j];
    out[j] = s;
}

// p -= sum_j c_j Q_j ; optional ||p||^2 partials (of the stored, rounded values)
template <typename T>
__global__ void __launch_bounds__(kThreads)
update_kernel(const T *__restrict__ Q, int64_t ldq, int m, const double *__restrict__ c,
              T *__restrict__ p, int64_t n, double *__restrict__ part)
{
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

template <typename T>
__global__ void scale_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t n,
                             const double *__restrict__ div, int is_norm2)
{
    const double d = is_norm2 ? sqrt(*div) : *div;
    const double f = (d > 0.0) ? 1.0 / d : 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride)
        dst[i] = (T)((double)src[i] * f);
}

__global__ void finalize_kernel(LanczosScalars *S, int i)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    S->alpha[i] = S->c1[i] + S->c2[i];
    S->beta[i] = sqrt(S->norm2);
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
ritz_kernel(T *__restrict__ Q, int64_t ldq, int m, const double *__restrict__ s, int64_t n,
            double *__restrict__ part)
{
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
                            double *partials, double *out, cudaStream_t st)
{
    const int g = grid_for(n);
    if (dtype == 0)
        multidot_kernel<double><<<g, kThreads, 0, st>>>((const double *)Q, ld, m, (const double *)p, n, partials);
    else
        multidot_kernel<float><<<g, kThreads, 0, st>>>((const float *)Q, ld, m, (const float *)p, n, partials);
    reduce_kernel<<<1, kMaxWindow, 0, st>>>(partials, g, m, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t update_launch(int dtype, const void *Q, int64_t ld, int m, const double *c, void *p,
                          int64_t n, double *partials, double *norm_out, cudaStream_t st)
{
    const int g = grid_for(n);
    double *part = norm_out ? partials : nullptr;
    if (dtype == 0)
        update_kernel<double><<<g, kThreads, 0, st>>>((const double *)Q, ld, m, c, (double *)p, n, part);
    else
        update_kernel<float><<<g, kThreads, 0, st>>>((const float *)Q, ld, m, c, (float *)p, n, part);
    if (norm_out) reduce_kernel<<<1, kMaxWindow, 0, st>>>(partials, g, 1, norm_out);
    count_launches((norm_out ? 2 : 1));
    return cudaGetLastError();
}

cudaError_t scale_launch(int dtype, const void *src, void *dst, int64_t n, const double *div,
                         int div_is_norm2, cudaStream_t st)
{
    const int g = grid_for(n);
    if (dtype == 0)
        scale_kernel<double><<<g, kThreads, 0, st>>>((const double *)src, (double *)dst, n, div, div_is_norm2);
    else
        scale_kernel<float><<<g, kThreads, 0, st>>>((const float *)src, (float *)dst, n, div, div_is_norm2);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t finalize_step_launch(LanczosScalars *S, int i, cudaStream_t st)
{
    finalize_kernel<<<1, 32, 0, st>>>(S, i);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t tridiag_launch(LanczosScalars *S, int m, cudaStream_t st)
{
    tridiag_kernel<<<1, 32, 0, st>>>(S, m);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t ritz_launch(int dtype, void *Q, int64_t ld, int m, const double *s, int64_t n,
                        double *partials, double *norm_out, cudaStream_t st)
{
    const int g = grid_for(n);
    if (dtype == 0)
        ritz_kernel<double><<<g, kThreads, 0, st>>>((double *)Q, ld, m, s, n, partials);
    else
        ritz_kernel<float><<<g, kThreads, 0, st>>>((float *)Q, ld, m, s, n, partials);
    reduce_kernel<<<1, kMaxWindow, 0, st>>>(partials, g, 1, norm_out);
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
    reduce_kernel<<<1, kMaxWindow, 0, st>>>(partials, g, 1, norm_out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace pd
