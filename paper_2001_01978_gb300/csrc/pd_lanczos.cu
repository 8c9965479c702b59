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
#include <cstdint>
#include <initializer_list>

namespace pd {
namespace {

constexpr int kThreads = 256;
constexpr int kGroup = 8;             // vectors handled per pass of a multi-vector kernel
// at most 4 CTAs per SM for the streaming kernels, and no more than the
// partial-sum buffers hold
inline int grid_cap()
{
    const int g = sm_count() * 4;
    return g < kMaxVecGrid ? g : kMaxVecGrid;
}

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ float fma_t<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <>
__device__ __forceinline__ double fma_t<double>(double a, double b, double c) { return fma(a, b, c); }

// ---- packs: W consecutive elements moved as one 16-byte access --------------
// W = 16 / sizeof(T) when every vector of a launch is 16-byte aligned, else 1.
// Pack c holds elements c*W .. c*W+W-1; the last pack of a vector whose length
// is not a multiple of W is read element by element (zero past the end) and
// written element by element, so n need not be a multiple of W.
template <typename T, int W>
struct Pack {
    T v[W];
};

template <typename T> struct Wide;
template <> struct Wide<float> { using type = float4; };
template <> struct Wide<double> { using type = double2; };

template <typename T, int W, bool RO>
__device__ __forceinline__ Pack<T, W> load_pack(const T *a, int64_t c, int64_t n)
{
    Pack<T, W> r;
    const int64_t e = c * W;
    if constexpr (W > 1) {
        static_assert(sizeof(T) * W == kPackBytes, "pack width");
        if (e + W <= n) {
            using V = typename Wide<T>::type;
            const V *pv = reinterpret_cast<const V *>(a) + c;
            const V t = RO ? __ldg(pv) : *pv;
            const T *tv = reinterpret_cast<const T *>(&t);
#pragma unroll
            for (int k = 0; k < W; ++k) r.v[k] = tv[k];
            return r;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) r.v[k] = (e + k < n) ? (RO ? __ldg(a + e + k) : a[e + k]) : T(0);
    return r;
}

template <typename T, int W>
__device__ __forceinline__ void store_pack(T *a, int64_t c, int64_t n, const Pack<T, W> &r)
{
    const int64_t e = c * W;
    if constexpr (W > 1) {
        if (e + W <= n) {
            using V = typename Wide<T>::type;
            V t;
            T *tv = reinterpret_cast<T *>(&t);
#pragma unroll
            for (int k = 0; k < W; ++k) tv[k] = r.v[k];
            reinterpret_cast<V *>(a)[c] = t;
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k)
        if (e + k < n) a[e + k] = r.v[k];
}

// The CTA-wide sums of a group of accumulators in one pass: every warp reduces
// each accumulator with shuffles and lane 0 keeps the warp's sums in shared
// memory; after one barrier thread u adds accumulator u's warp sums in warp
// order (a fixed order) and writes out[u].  nvalid (CTA-uniform) accumulators
// are used; shg holds kGroup * kThreads / 32 doubles.  Ends with a barrier, so
// shg can be reused at once.
template <typename T>
__device__ __forceinline__ void block_reduce_group(const DotAcc<T> (&acc)[kGroup], int nvalid, double *shg,
                                                   double *out)
{
    constexpr int NW = kThreads / 32;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < kGroup; ++u) {
        if (u < nvalid) {
            const double v = warp_reduce(acc[u]);
            if (lane == 0) shg[u * NW + w] = v;
        }
    }
    __syncthreads();
    if ((int)threadIdx.x < nvalid) {
        double sum = 0.0;
        for (int i = 0; i < NW; ++i) sum += shg[threadIdx.x * NW + i];
        out[threadIdx.x] = sum;
    }
    __syncthreads();
}

// Lanczos step bookkeeping (Algorithm 2): alpha_i = alpha + c_i (the second
// Gram-Schmidt pass corrects the recurrence's alpha), beta_i = ||p||; a beta_i
// below 1e-13 of the running matrix-norm estimate ends the cycle (an invariant
// subspace, or a NaN).
__device__ __forceinline__ void finalize_step(LanczosScalars *S, int i, double norm2)
{
    if (S->broken) return;
    const double a = S->c1[0] + S->c2[i];
    const double b = sqrt(norm2);
    S->alpha[i] = a;
    S->beta[i] = b;
    const double row = fabs(a) + b + (i > 0 ? S->beta[i - 1] : 0.0);
    const double tn = fmax(S->tnorm, row);
    S->tnorm = tn;
    S->used = i + 1;
    if (!(b > 1e-13 * tn)) S->broken = 1;
}

// out[j] = Q_j^T p for j < m (partials per CTA; with a ticket the last CTA adds
// them).  NG vectors per pass: 1 for a single dot, so that no predicated-off
// multiply-adds are issued (FP64 ones occupy GB300's small FP64 pipe).
template <typename T, int W, int NG = kGroup>
__global__ void __launch_bounds__(kThreads)
dots_kernel(const T *__restrict__ Q, int64_t ldq, int m, const T *__restrict__ p, int64_t n,
            double *__restrict__ part, double *__restrict__ out, unsigned long long *ticket,
            const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ double shg[kGroup * (kThreads / 32)];
    const int64_t nc = (n + W - 1) / W;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t c0 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    for (int j0 = 0; j0 < m; j0 += NG) {
        DotAcc<T> acc[kGroup];
        for (int64_t c = c0; c < nc; c += stride) {
            const Pack<T, W> pv = load_pack<T, W, true>(p, c, n);
            Pack<T, W> q[kGroup];
#pragma unroll
            for (int u = 0; u < NG; ++u)
                if (j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq, c, n);
#pragma unroll
            for (int u = 0; u < NG; ++u)
                if (j0 + u < m)
#pragma unroll
                    for (int k = 0; k < W; ++k) acc[u].add(q[u].v[k], pv.v[k]);
        }
        block_reduce_group<T>(acc, min(NG, m - j0), shg, part + (int64_t)blockIdx.x * kMaxWindow + j0);
    }
    if (ticket && arrive_last(ticket)) reduce_partials(part, gridDim.x, m, out);
}

// Lanczos recurrence fused with the projections of one Gram-Schmidt pass:
//   p <- p - alpha q_i - beta_{i-1} q_{i-1}   (Algorithm 2; alpha = S->c1[0])
//   out[j] = Q_j^T p for j <= i (after the update)
// Every pack is visited by the same thread in every group, so the groups after
// the first read back this thread's own updated values.
template <typename T, int W>
__global__ void __launch_bounds__(kThreads, 3)
recur_project_kernel(const T *__restrict__ Q, int64_t ldq, int i, const LanczosScalars *__restrict__ S,
                     T *__restrict__ p, int64_t n, double *__restrict__ part, double *__restrict__ out,
                     unsigned long long *ticket, const int *__restrict__ skip)
{
    if (skip && *skip) return;
    __shared__ double shg[kGroup * (kThreads / 32)];
    const int m = i + 1;
    const T a = (T)S->c1[0];
    const T b = (T)(i > 0 ? S->beta[i - 1] : 0.0);
    const T *qi = Q + (int64_t)i * ldq;
    const T *qm = Q + (int64_t)(i > 0 ? i - 1 : 0) * ldq;
    T cr[kGroup];                                 // recurrence coefficients of group 0
#pragma unroll
    for (int u = 0; u < kGroup; ++u) cr[u] = (u == i) ? a : (u == i - 1) ? b : T(0);
    const int64_t nc = (n + W - 1) / W;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    const int64_t c0 = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    for (int j0 = 0; j0 < m; j0 += kGroup) {
        DotAcc<T> acc[kGroup];
        for (int64_t c = c0; c < nc; c += stride) {
            Pack<T, W> v = load_pack<T, W, false>(p, c, n);
            Pack<T, W> q[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq, c, n);
            if (j0 == 0) {
                if (i < kGroup) {
                    // q_i and q_{i-1} are packs of this group: one sweep over the
                    // group, highest index first, whose coefficients vanish except
                    // at i (alpha) and i-1 (beta), so q_i is applied before q_{i-1}
#pragma unroll
                    for (int u = kGroup - 1; u >= 0; --u)
                        if (u <= i)
#pragma unroll
                            for (int k = 0; k < W; ++k) v.v[k] = fma_t<T>(-cr[u], q[u].v[k], v.v[k]);
                } else {
                    const Pack<T, W> x = load_pack<T, W, true>(qi, c, n);
                    const Pack<T, W> y = load_pack<T, W, true>(qm, c, n);
#pragma unroll
                    for (int k = 0; k < W; ++k) v.v[k] = fma_t<T>(-b, y.v[k], fma_t<T>(-a, x.v[k], v.v[k]));
                }
                store_pack<T, W>(p, c, n, v);
            }
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m)
#pragma unroll
                    for (int k = 0; k < W; ++k) acc[u].add(q[u].v[k], v.v[k]);
        }
        block_reduce_group<T>(acc, min(kGroup, m - j0), shg, part + (int64_t)blockIdx.x * kMaxWindow + j0);
    }
    if (ticket && arrive_last(ticket)) reduce_partials(part, gridDim.x, m, out);
}

// out[j] = sum_b part[b*kMaxWindow + j] in one CTA (launches without a ticket)
__global__ void reduce_kernel(const double *__restrict__ part, int nb, int m, double *__restrict__ out,
                              const int *__restrict__ skip)
{
    if (skip && *skip) return;
    reduce_partials(part, nb, m, out);
}

inline void reduce(const double *part, int nb, int m, double *out, cudaStream_t st, const int *skip = nullptr)
{
    reduce_kernel<<<1, 256, 0, st>>>(part, nb, m, out, skip);
    count_launches(1);
}

// p -= sum_j c_j Q_j in the storage type (FP32 FMAs for float: the result is
// stored in FP32 anyway, and the second Gram-Schmidt pass removes what this
// rounding leaves along Q); optional ||p||^2 of the stored values; optional
// step bookkeeping by the last CTA
template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
update_kernel(const T *__restrict__ Q, int64_t ldq, int m, const double *__restrict__ c,
              T *__restrict__ p, int64_t n, double *__restrict__ part, double *__restrict__ norm_out,
              unsigned long long *ticket, const int *__restrict__ skip, LanczosScalars *fin, int fin_i)
{
    if (skip && *skip) return;
    __shared__ T sc[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < m; j += kThreads) sc[j] = (T)c[j];
    __syncthreads();
    DotAcc<T> nrm;
    const int64_t nc = (n + W - 1) / W;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < nc; e += stride) {
        Pack<T, W> v = load_pack<T, W, false>(p, e, n);
        for (int j0 = 0; j0 < m; j0 += kGroup) {
            Pack<T, W> q[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq, e, n);
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m)
#pragma unroll
                    for (int k = 0; k < W; ++k) v.v[k] = fma_t<T>(-sc[j0 + u], q[u].v[k], v.v[k]);
        }
        store_pack<T, W>(p, e, n, v);
#pragma unroll
        for (int k = 0; k < W; ++k) nrm.add(v.v[k], v.v[k]);
    }
    if (norm_out) {
        const double s = block_reduce(nrm, sh);
        if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = s;
        if (ticket && arrive_last(ticket)) {
            const double nn = reduce_partials(part, gridDim.x, 1, norm_out);
            if (fin && threadIdx.x == 0) finalize_step(fin, fin_i, nn);
        }
    }
}

// dst = src * f with f = 1 / *div (or 1 / sqrt(*div)); src may be dst
template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
scale_kernel(const T *src, T *dst, int64_t n, const double *__restrict__ div, int is_norm2,
             const int *__restrict__ skip)
{
    if (skip && *skip) return;
    const double d = is_norm2 ? sqrt(*div) : *div;
    const T f = (d > 0.0) ? (T)(1.0 / d) : T(0);
    const int64_t nc = (n + W - 1) / W;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < nc; c += stride) {
        Pack<T, W> v = load_pack<T, W, false>(src, c, n);
#pragma unroll
        for (int k = 0; k < W; ++k) v.v[k] = v.v[k] * f;
        store_pack<T, W>(dst, c, n, v);
    }
}

// ---- one Lanczos step after the product, in one cooperative launch ---------
// The recurrence, one full Gram-Schmidt pass against every stored vector, the
// norm and the scaling into the next basis vector (Algorithm 2, Sec. 3.4) with
// two grid-wide barriers in between instead of three launches.  CTA b owns
// packs [b*slice, (b+1)*slice) of every vector; with SMEM its part of p stays in
// shared memory from the recurrence to the scaling, so p is read once and never
// written.  Every CTA adds the CTAs' partial sums in the same fixed order, so
// all of them hold bit-identical coefficients.
constexpr int kStepThreads = 512;
constexpr int kStepWarps = kStepThreads / 32;
constexpr unsigned kBarPolls = 1u << 24;      // x >= 64 ns: a barrier gives up after about a second

// Dot-product accumulator of the step kernel, one pack at a time.  FP32: the
// pack's W products are summed with FP32 FMAs and the pack sum is added to a
// float-float total with Knuth's TwoSum (10 instructions per pack of 4 instead
// of 32 for exact products).  The rounding of a pack sum is relative to that
// pack's own products, so it stays far below the FP32 rounding of the stored
// vectors.  FP64: FP64 FMAs.
template <typename T> struct PackAcc;
template <> struct PackAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    template <int W>
    __device__ __forceinline__ void add(const Pack<float, W> &a, const Pack<float, W> &b)
    {
        float s = a.v[0] * b.v[0];
#pragma unroll
        for (int k = 1; k < W; ++k) s = fmaf(a.v[k], b.v[k], s);
        const float t = hi + s;
        const float z = t - hi;
        lo += (hi - (t - z)) + (s - z);
        hi = t;
    }
};
template <> struct PackAcc<double> {
    double v = 0.0;
    template <int W>
    __device__ __forceinline__ void add(const Pack<double, W> &a, const Pack<double, W> &b)
    {
#pragma unroll
        for (int k = 0; k < W; ++k) v = fma(a.v[k], b.v[k], v);
    }
};

// float-float (FP32) or FP64 partial sums of the step kernel
template <typename T> struct StepRed;
template <> struct StepRed<float> {
    using P = float2;
    static __device__ __forceinline__ P zero() { return make_float2(0.0f, 0.0f); }
    static __device__ __forceinline__ P from(const PackAcc<float> &a) { return make_float2(a.hi, a.lo); }
    static __device__ __forceinline__ void add(P &a, P b) { ff_add(a.x, a.y, b.x, b.y); }
    static __device__ __forceinline__ P xor_shfl(P a, int o)
    {
        return make_float2(__shfl_xor_sync(0xffffffffu, a.x, o), __shfl_xor_sync(0xffffffffu, a.y, o));
    }
    static __device__ __forceinline__ double value(P a) { return (double)a.x + (double)a.y; }
};
template <> struct StepRed<double> {
    using P = double;
    static __device__ __forceinline__ P zero() { return 0.0; }
    static __device__ __forceinline__ P from(const PackAcc<double> &a) { return a.v; }
    static __device__ __forceinline__ void add(P &a, P b) { a += b; }
    static __device__ __forceinline__ P xor_shfl(P a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    static __device__ __forceinline__ double value(P a) { return a; }
};

template <typename R>
__device__ __forceinline__ typename R::P warp_allsum(typename R::P s)
{
    for (int o = 16; o > 0; o >>= 1) R::add(s, R::xor_shfl(s, o));
    return s;
}

// Grid-wide barrier of a cooperative launch (all CTAs resident).  Thread 0
// reads the generation before it arrives (acquire loads, release stores); the
// last CTA to arrive resets the count and opens the next generation.  A wait
// longer than kBarPolls polls sets gb->err and returns false (the caller
// returns at once; the other CTAs then give up at this barrier or the next).
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *a)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(unsigned int *a, unsigned int v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(GridBar *gb, int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int g = ld_acquire_u32(&gb->gen);
        __threadfence();                                     // release this CTA's writes
        if (atomicAdd(&gb->count, 1u) == gridDim.x - 1u) {
            gb->count = 0u;
            st_release_u32(&gb->gen, g + 1u);
        } else {
            unsigned int polls = 0;
            while (ld_acquire_u32(&gb->gen) == g) {
                if (++polls > kBarPolls) {
                    atomicExch(&gb->err, 1);
                    ok = 0;
                    break;
                }
                if (polls > 64) __nanosleep(32);
            }
        }
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// the packs c of the group's vectors Q_j0 .. Q_{j0+KG-1} that exist (j < m)
template <typename T, int W, int KG>
__device__ __forceinline__ void load_group(Pack<T, W> (&q)[KG], const T *__restrict__ Q, int64_t ldq, int j0,
                                           int m, int64_t c, int64_t n)
{
#pragma unroll
    for (int u = 0; u < KG; ++u)
        if (KG == 1 || j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq, c, n);
}

// Ownership: the packs form chunks of kStepThreads; CTA b owns the K
// consecutive chunks b*K .. b*K + K - 1, thread t pack t of each.  Local pack
// slot (chunk l of the CTA, thread t) = l * kStepThreads + t.
// KG: vectors per group pass (1, 2, 4 or 8, chosen per launch so that the
// last group issues few predicated-off multiply-adds)
template <typename T, int W, bool SMEM, int KG>
__global__ void __launch_bounds__(kStepThreads, 1)
step_kernel(const T *__restrict__ Q, int64_t ldq, int i, LanczosScalars *S, T *p, int64_t n,
            typename StepRed<T>::P *part, GridBar *gb, T *qnext)
{
    using R = StepRed<T>;
    using P = typename R::P;
    extern __shared__ __align__(16) unsigned char step_smem[];
    Pack<T, W> *sv = reinterpret_cast<Pack<T, W> *>(step_smem);   // this CTA's packs of p (SMEM)
    __shared__ P wpart[kStepWarps][kMaxWindow];
    __shared__ double sc[kMaxWindow];
    __shared__ T scT[kMaxWindow];
    __shared__ T s_ab[3];                         // alpha, beta_{i-1}, 1 / beta_i in the storage type
    __shared__ double s_in[3];                    // alpha, beta_{i-1}, tnorm as the launch found them
    __shared__ int s_ok, s_brk;
    if (S->broken) return;                        // uniform: nothing in this launch writes it before the barriers
    const int m = i + 1;
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    // the FP64 scalars once per CTA (GB300 runs FP64 at a small fraction of
    // FP32), read before the first barrier: block 0 rewrites tnorm after the last
    if (tid == 0) {
        s_in[0] = S->c1[0];
        s_in[1] = i > 0 ? S->beta[i - 1] : 0.0;
        s_in[2] = S->tnorm;
        s_ab[0] = (T)s_in[0];
        s_ab[1] = (T)s_in[1];
    }
    __syncthreads();
    const T a = s_ab[0], b = s_ab[1];
    const T *qi = Q + (int64_t)i * ldq;
    const T *qm = Q + (int64_t)(i > 0 ? i - 1 : 0) * ldq;
    const int64_t nc = (n + W - 1) / W;
    const int64_t nchunk = (nc + kStepThreads - 1) / kStepThreads;
    const int64_t G = gridDim.x;
    const int64_t K = (nchunk + G - 1) / G;
    const int64_t first = (int64_t)blockIdx.x * K;
    const int64_t mine = first < nchunk ? (nchunk - first < K ? nchunk - first : K) : 0;   // chunks of this CTA
    const int ng = (m + KG - 1) / KG;
    auto pack_of = [&](int64_t l) { return (first + l) * kStepThreads + tid; };

    // phase 1: p <- p - alpha q_i - beta_{i-1} q_{i-1}; c_j = Q_j^T p (j <= i).
    // Two chunks per iteration, all their loads issued before the first use.
    for (int g = 0; g < ng; ++g) {
        const int j0 = g * KG;
        PackAcc<T> acc[KG];
        for (int64_t l = 0; l < mine; l += 2) {
            const int64_t c0 = pack_of(l), c1 = pack_of(l + 1);
            const bool ok0 = c0 < nc, ok1 = l + 1 < mine && c1 < nc;
            Pack<T, W> v[2], q[2][KG];
            if (g == 0) {
                Pack<T, W> x[2], y[2];
                if (ok0) {
                    v[0] = load_pack<T, W, false>(p, c0, n);
                    x[0] = load_pack<T, W, true>(qi, c0, n);
                    y[0] = load_pack<T, W, true>(qm, c0, n);
                    load_group<T, W, KG>(q[0], Q, ldq, j0, m, c0, n);
                }
                if (ok1) {
                    v[1] = load_pack<T, W, false>(p, c1, n);
                    x[1] = load_pack<T, W, true>(qi, c1, n);
                    y[1] = load_pack<T, W, true>(qm, c1, n);
                    load_group<T, W, KG>(q[1], Q, ldq, j0, m, c1, n);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!(h == 0 ? ok0 : ok1)) continue;
#pragma unroll
                    for (int k = 0; k < W; ++k)
                        v[h].v[k] = fma_t<T>(-b, y[h].v[k], fma_t<T>(-a, x[h].v[k], v[h].v[k]));
                    if (SMEM) sv[(l + h) * kStepThreads + tid] = v[h];
                    else store_pack<T, W>(p, h == 0 ? c0 : c1, n, v[h]);
                }
            } else {
                if (ok0) {
                    v[0] = SMEM ? sv[l * kStepThreads + tid] : load_pack<T, W, false>(p, c0, n);
                    load_group<T, W, KG>(q[0], Q, ldq, j0, m, c0, n);
                }
                if (ok1) {
                    v[1] = SMEM ? sv[(l + 1) * kStepThreads + tid] : load_pack<T, W, false>(p, c1, n);
                    load_group<T, W, KG>(q[1], Q, ldq, j0, m, c1, n);
                }
            }
            if (ok0) {
#pragma unroll
                for (int u = 0; u < KG; ++u)
                    if (j0 + u < m) acc[u].add(q[0][u], v[0]);
            }
            if (ok1) {
#pragma unroll
                for (int u = 0; u < KG; ++u)
                    if (j0 + u < m) acc[u].add(q[1][u], v[1]);
            }
        }
#pragma unroll
        for (int u = 0; u < KG; ++u)
            if (j0 + u < m) {
                const P s = warp_allsum<R>(R::from(acc[u]));
                if (lane == 0) wpart[w][j0 + u] = s;
            }
    }
    __syncthreads();
    if (tid < m) {
        P s = R::zero();
        for (int x = 0; x < kStepWarps; ++x) R::add(s, wpart[x][tid]);
        part[(int64_t)blockIdx.x * kMaxWindow + tid] = s;
    }
    if (!grid_sync(gb, &s_ok)) return;
    // every CTA adds the CTAs' partial sums in the same order
    for (int j = w; j < m; j += kStepWarps) {
        P s = R::zero();
        for (int x = lane; x < (int)G; x += 32) R::add(s, __ldcg(part + (int64_t)x * kMaxWindow + j));
        s = warp_allsum<R>(s);
        if (lane == 0) {
            const double c = R::value(s);
            sc[j] = c;
            scT[j] = (T)c;
        }
    }
    __syncthreads();

    // phase 2: p <- p - sum_j c_j Q_j, the groups in reverse (the vectors phase 1
    // read last are the likeliest still in L2), then ||p||^2
    PackAcc<T> nrm;
    for (int g = ng - 1; g >= 0; --g) {
        const int j0 = g * KG;
        T cg[KG];
#pragma unroll
        for (int u = 0; u < KG; ++u) cg[u] = (j0 + u < m) ? scT[j0 + u] : T(0);
        for (int64_t l = 0; l < mine; l += 2) {
            const int64_t c0 = pack_of(l), c1 = pack_of(l + 1);
            const bool ok0 = c0 < nc, ok1 = l + 1 < mine && c1 < nc;
            Pack<T, W> v[2], q[2][KG];
            if (ok0) {
                v[0] = SMEM ? sv[l * kStepThreads + tid] : load_pack<T, W, false>(p, c0, n);
                load_group<T, W, KG>(q[0], Q, ldq, j0, m, c0, n);
            }
            if (ok1) {
                v[1] = SMEM ? sv[(l + 1) * kStepThreads + tid] : load_pack<T, W, false>(p, c1, n);
                load_group<T, W, KG>(q[1], Q, ldq, j0, m, c1, n);
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h == 0 ? ok0 : ok1)) continue;
#pragma unroll
                for (int u = 0; u < KG; ++u)
                    if (j0 + u < m)
#pragma unroll
                        for (int k = 0; k < W; ++k) v[h].v[k] = fma_t<T>(-cg[u], q[h][u].v[k], v[h].v[k]);
                if (g == 0) nrm.add(v[h], v[h]);
                if (SMEM) sv[(l + h) * kStepThreads + tid] = v[h];
                else store_pack<T, W>(p, h == 0 ? c0 : c1, n, v[h]);
            }
        }
    }
    {
        const P s = warp_allsum<R>(R::from(nrm));
        if (lane == 0) wpart[w][0] = s;
    }
    __syncthreads();
    P *npart = part + G * kMaxWindow;
    if (tid == 0) {
        P s = R::zero();
        for (int x = 0; x < kStepWarps; ++x) R::add(s, wpart[x][0]);
        npart[blockIdx.x] = s;
    }
    if (!grid_sync(gb, &s_ok)) return;
    // the norm, and the step bookkeeping (the arithmetic of finalize_step) in one
    // thread per CTA, every CTA alike
    if (w == 0) {
        P s = R::zero();
        for (int x = lane; x < (int)G; x += 32) R::add(s, __ldcg(npart + x));
        s = warp_allsum<R>(s);
        if (lane == 0) {
            const double norm2 = R::value(s);
            const double ai = s_in[0] + sc[i];
            const double bi = sqrt(norm2);
            const double tn = fmax(s_in[2], fabs(ai) + bi + s_in[1]);
            const int brk = !(bi > 1e-13 * tn);
            s_brk = brk;
            s_ab[2] = brk ? T(0) : (T)(1.0 / bi);
            if (blockIdx.x == 0) {
                S->norm2 = norm2;
                S->alpha[i] = ai;
                S->beta[i] = bi;
                S->tnorm = tn;
                S->used = i + 1;
                if (brk) S->broken = 1;
            }
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && tid < m) S->c2[tid] = sc[tid];
    // phase 3: q_{i+1} = p / beta_i
    if (s_brk || !qnext) return;
    const T f = s_ab[2];
    for (int64_t l = 0; l < mine; ++l) {
        const int64_t cc = pack_of(l);
        if (cc >= nc) continue;
        Pack<T, W> v = SMEM ? sv[l * kStepThreads + tid] : load_pack<T, W, false>(p, cc, n);
#pragma unroll
        for (int k = 0; k < W; ++k) v.v[k] = v.v[k] * f;
        store_pack<T, W>(qnext, cc, n, v);
    }
}

__global__ void quotient_kernel(const double *num, const double *den, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *out = *num / *den;
}

__global__ void cycle_reset_kernel(LanczosScalars *S)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    S->used = 0;
    S->broken = 0;
    S->tnorm = 0.0;
}

// ---- symmetric tridiagonal eigenproblem (one warp) --------------------------
// Number of eigenvalues below x: sign changes of the characteristic-polynomial
// sequence p_0 = 1, p_1 = a_0 - x, p_i = (a_{i-1} - x) p_{i-1} - b2_{i-2} p_{i-2}
// (Sturm), evaluated without divisions on a matrix scaled to entries <= 1 so that
// no p_i leaves the double range for m <= 64.  A zero p_i takes the sign opposite
// to p_{i-1}.
template <typename R>
__device__ __forceinline__ int sturm_count(const R *a, const R *b2, int m, R x)
{
    R pm2 = R(1), pm1 = a[0] - x;
    if (pm1 == R(0)) pm1 = -R(1e-30);
    int cnt = pm1 < R(0);
    for (int i = 1; i < m; ++i) {
        R p = (a[i] - x) * pm1 - b2[i - 1] * pm2;
        if (p == R(0)) p = pm1 < R(0) ? R(1e-30) : -R(1e-30);
        cnt += (p < R(0)) != (pm1 < R(0));
        pm2 = pm1;
        pm1 = p;
    }
    return cnt;
}

// j-th smallest eigenvalue (j = 1, 2, ...) inside [lo, hi] by 33-way multisection
// across the warp, until the bracket is `rel` wide (relative) or stops shrinking
template <typename R>
__device__ void multisect(const R *a, const R *b2, int m, int j, R &lo, R &hi, R rel)
{
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < 64; ++it) {
        const R w = hi - lo;
        const R mag = fabs(lo) > fabs(hi) ? fabs(lo) : fabs(hi);
        if (w <= rel * mag || w <= (sizeof(R) == 4 ? R(FLT_MIN) : R(DBL_MIN))) break;
        const R xl = lo + w * R(lane + 1) / R(33);
        const int c = sturm_count<R>(a, b2, m, xl);
        const unsigned below = __ballot_sync(0xffffffffu, c < j);    // eigenvalue j lies above xl
        const int nb = __popc(below);                                 // the points below are a prefix
        const R new_lo = nb > 0 ? __shfl_sync(0xffffffffu, xl, nb - 1) : lo;
        const R new_hi = nb < 32 ? __shfl_sync(0xffffffffu, xl, nb < 32 ? nb : 31) : hi;
        if (new_lo == lo && new_hi == hi) break;
        lo = new_lo;
        hi = new_hi;
    }
}

// ---- costs on GB300 that shape the code below ---------------------------------
// A dependent FP64 FMA takes about 64 cycles and an FP64 division about 650,
// against 4.5 and 64 for FP32.  So the small eigenproblem does its searching
// in FP32, keeps FP64 for the final digits, spreads element-wise FP64 work
// over the lanes, and replaces each FP64 division on a serial chain by one
// reciprocal formed from an FP32 seed and two Newton-Raphson steps
// r <- r + r (1 - x r) (the error squares at each step: 2^-22 -> 2^-44 -> 2^-88).

__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float rsqrt_approx(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// 1 / x for 1e-30 <= |x| <= 1e30
__device__ __forceinline__ double rcp64(double x)
{
    double r = (double)rcp_approx((float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return r;
}

// pivot magnitudes below `tiny` are raised to it (sign kept; zero -> +tiny)
template <typename R>
__device__ __forceinline__ R guard_pivot(R c, R tiny)
{
    return fabs(c) >= tiny ? c : (c < R(0) ? -tiny : tiny);
}

// Solve (T - theta I) z = r for a symmetric tridiagonal T (diagonal a, off-
// diagonal b) by Gaussian elimination with partial pivoting (rows i and i+1 may
// swap; the upper factor then has two superdiagonals).  One reciprocal per row
// (rcp64 in FP64, rcp.approx in FP32); pivots below 1e-30 are raised to it.
template <typename R>
__device__ void tridiag_solve(const R *a, const R *b, int m, R theta, R *r, R *u0inv, R *u1, R *u2)
{
    const R tiny = R(1e-30);
    R c0 = a[0] - theta, c1 = (m > 1 ? b[0] : R(0)), c2 = R(0);
    for (int i = 0; i < m - 1; ++i) {
        R n0 = b[i], n1 = a[i + 1] - theta, n2 = (i + 2 < m ? b[i + 1] : R(0));
        if (fabs(n0) > fabs(c0)) {      // swap rows i and i+1
            R t;
            t = c0; c0 = n0; n0 = t;
            t = c1; c1 = n1; n1 = t;
            t = c2; c2 = n2; n2 = t;
            t = r[i]; r[i] = r[i + 1]; r[i + 1] = t;
        }
        c0 = guard_pivot<R>(c0, tiny);
        R inv;
        if constexpr (sizeof(R) == 8) inv = rcp64(c0);
        else inv = rcp_approx(c0);
        const R mu = n0 * inv;
        u0inv[i] = inv; u1[i] = c1; u2[i] = c2;
        r[i + 1] -= mu * r[i];
        c0 = n1 - mu * c1;
        c1 = n2 - mu * c2;
        c2 = R(0);
    }
    c0 = guard_pivot<R>(c0, tiny);
    if constexpr (sizeof(R) == 8) u0inv[m - 1] = rcp64(c0);
    else u0inv[m - 1] = rcp_approx(c0);
    u1[m - 1] = R(0); u2[m - 1] = R(0);
    for (int i = m - 1; i >= 0; --i) {
        R t = r[i];
        if (i + 1 < m) t -= u1[i] * r[i + 1];
        if (i + 2 < m) t -= u2[i] * r[i + 2];
        r[i] = t * u0inv[i];
    }
}

// z <- z / ||z|| (one lane; z first scaled by its largest magnitude, so the sum
// of squares lies in [1, m] and an FP32 seed + two Newton steps give 1/sqrt)
template <typename R>
__device__ void normalise(R *z, int m)
{
    R big = R(0);
    for (int i = 0; i < m; ++i) big = fmax(big, fabs(z[i]));
    if (!(big > R(0)) || !isfinite(big)) {        // degenerate: the first unit vector
        for (int i = 0; i < m; ++i) z[i] = i == 0 ? R(1) : R(0);
        return;
    }
    R sc;
    if constexpr (sizeof(R) == 8) sc = rcp64(big);
    else sc = rcp_approx(big);
    R nrm = R(0);
    for (int i = 0; i < m; ++i) {
        z[i] *= sc;
        nrm += z[i] * z[i];
    }
    R y = (R)rsqrt_approx((float)nrm);
    if constexpr (sizeof(R) == 8) {
        y = y * fma(-0.5 * nrm * y, y, 1.5);
        y = y * fma(-0.5 * nrm * y, y, 1.5);
    }
    for (int i = 0; i < m; ++i) z[i] *= y;
}

// Gershgorin bound of tridiag(alpha, beta) rounded up to a power of two, so
// that scaling by it is exact in FP32 and FP64: lane k takes rows k, k+32.
// Returns 2^e in every lane (1 for a zero matrix).
__device__ __forceinline__ float gershgorin_pow2(const double *alpha, const double *beta, int m)
{
    const int lane = threadIdx.x & 31;
    float g = 0.0f;
    for (int k = lane; k < m; k += 32) {
        const float rad = (k + 1 < m ? fabsf((float)beta[k]) : 0.0f) + (k > 0 ? fabsf((float)beta[k - 1]) : 0.0f);
        g = fmaxf(g, fabsf((float)alpha[k]) + rad);
    }
    for (int o = 16; o > 0; o >>= 1) g = fmaxf(g, __shfl_xor_sync(0xffffffffu, g, o));
    if (!(g > 0.0f) || !isfinite(g)) return 1.0f;
    int e;
    frexpf(g * 1.0000002f, &e);                  // g * (1 + 2 ulp) <= 2^e
    return ldexpf(1.0f, e);
}

// p_m, p_m' and p_{m-1}, p_{m-1}' at x for the scaled matrix (diagonal a,
// squared off-diagonal b2), p_k = (a_{k-1} - x) p_{k-1} - b2_{k-2} p_{k-2}:
// no divisions, |p_k| <= 2.25^k.  One lane.
struct CharPoly {
    double pm, dpm, pm1, dpm1;
};
__device__ __forceinline__ CharPoly char_poly(const double *a, const double *b2, int m, double x)
{
    double p0 = 1.0, p1 = a[0] - x, d0 = 0.0, d1 = -1.0;
    for (int k = 1; k < m; ++k) {
        const double am = a[k] - x;
        const double p2 = fma(am, p1, -b2[k - 1] * p0);
        const double d2 = fma(am, d1, fma(-b2[k - 1], d0, -p1));
        p0 = p1; p1 = p2; d0 = d1; d1 = d2;
    }
    return CharPoly{p1, d1, p0, d0};
}

// Newton steps x <- x - p_m(x) / p_m'(x) for the lowest eigenvalue from the
// midpoint of an FP32 bracket [lo, hi] (one lane).  `evals` evaluations; cp
// holds the last one (at the returned x, before its own step).  False when a
// step leaves the bracket widened by 1e-6 or a value is not finite.
__device__ bool newton_lowest(const double *a, const double *b2, int m, float lo, float hi, int evals, double &x,
                              CharPoly &cp)
{
    const double wlo = (double)lo - 1e-6, whi = (double)hi + 1e-6;
    x = 0.5 * ((double)lo + (double)hi);
    for (int it = 0; it < evals; ++it) {
        cp = char_poly(a, b2, m, x);
        if (!(fabs(cp.dpm) >= 1e-30 && fabs(cp.dpm) <= 1e30) || !isfinite(cp.pm)) return false;
        if (it + 1 == evals) return true;
        const double xn = x - cp.pm * rcp64(cp.dpm);
        if (!(xn >= wlo && xn <= whi)) return false;
        x = xn;
    }
    return true;
}

// Lowest two eigenvalues and the lowest eigenvector of the m x m symmetric
// tridiagonal matrix (alpha, beta), computed by one warp.  Work arrays in
// shared memory (kMaxWindow doubles each).  Steps: exact power-of-two scaling;
// FP32 multisection brackets of the two lowest eigenvalues; Newton steps on the
// characteristic polynomial in FP64 for the lowest (FP64 multisection if they
// leave the bracket); two FP32 inverse iterations, then one in FP64 at the
// refined eigenvalue, for its eigenvector.
__device__ void tridiag_warp(const double *alpha, const double *beta, int m, double *theta_out, double *s_out,
                             double *a, double *b, double *b2, double *z, double *u0, double *u1, double *u2)
{
    const int lane = threadIdx.x & 31;
    const float scf = gershgorin_pow2(alpha, beta, m);
    const double scale = (double)scf, inv = 1.0 / (double)scf;      // exact powers of two
    float *af = reinterpret_cast<float *>(u0);
    float *bf = af + kMaxWindow;
    float *b2f = reinterpret_cast<float *>(u1);
    float *zf = b2f + kMaxWindow;
    for (int i = lane; i < m; i += 32) {
        a[i] = alpha[i] * inv;
        b[i] = (i + 1 < m) ? beta[i] * inv : 0.0;
        b2[i] = b[i] * b[i];
        af[i] = (float)a[i];
        bf[i] = (float)b[i];
        b2f[i] = (float)b2[i];
    }
    __syncwarp();
    if (m == 1) {
        if (lane == 0) { theta_out[0] = alpha[0]; theta_out[1] = INFINITY; s_out[0] = 1.0; }
        __syncwarp();
        return;
    }
    // FP32 brackets of the two lowest eigenvalues (entries are within [-1, 1])
    float lo1 = -1.25f, hi1 = 1.25f, lo2 = -1.25f, hi2 = 1.25f;
    multisect<float>(af, b2f, m, 1, lo1, hi1, 4e-7f);
    multisect<float>(af, b2f, m, 2, lo2, hi2, 4e-7f);
    const double wlo = (double)lo1 - 1e-6, whi = (double)hi1 + 1e-6;
    // three Newton steps in FP64 from the FP32 bracket (the error squares each
    // step: 4e-7 -> 1e-13 -> 1e-26), the last step taken from the last evaluation
    int ok = 0;
    double t1 = 0.0;
    if (lane == 0) {
        CharPoly cp;
        ok = newton_lowest(a, b2, m, lo1, hi1, 3, t1, cp);
        if (ok) {
            const double xn = t1 - cp.pm * rcp64(cp.dpm);
            ok = xn >= wlo && xn <= whi;
            t1 = xn;
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    t1 = __shfl_sync(0xffffffffu, t1, 0);
    if (!ok) {                                     // FP64 multisection from the widened bracket
        double lo = wlo, hi = whi;
        if (sturm_count<double>(a, b2, m, lo) >= 1) lo = -1.25;
        if (sturm_count<double>(a, b2, m, hi) < 1) hi = 1.25;
        multisect<double>(a, b2, m, 1, lo, hi, 2.0 * DBL_EPSILON);
        t1 = 0.5 * (lo + hi);
    }
    const double t2 = 0.5 * ((double)lo2 + (double)hi2);
    __syncwarp();
    if (lane == 0) {
        // eigenvector: two FP32 inverse iterations from (1, ..., 1) at the FP32
        // eigenvalue, then one FP64 iteration at the refined one
        const float t1f = (float)t1;
        float *u0f = reinterpret_cast<float *>(u2), *u1f = u0f + kMaxWindow;
        float *u2f = reinterpret_cast<float *>(b2) ;   // b2 is no longer needed
        for (int i = 0; i < m; ++i) zf[i] = 1.0f;
        for (int it = 0; it < 2; ++it) {
            tridiag_solve<float>(af, bf, m, t1f, zf, u0f, u1f, u2f);
            normalise<float>(zf, m);
        }
        for (int i = 0; i < m; ++i) z[i] = (double)zf[i];
        tridiag_solve<double>(a, b, m, t1, z, u0, u1, u2);
        normalise<double>(z, m);
        double big = 0.0; int ib = 0;                 // fix the sign: largest component positive
        for (int i = 0; i < m; ++i) if (fabs(z[i]) > big) { big = fabs(z[i]); ib = i; }
        const double sg = z[ib] < 0.0 ? -1.0 : 1.0;
        for (int i = 0; i < m; ++i) s_out[i] = sg * z[i];
        theta_out[0] = t1 * scale;
        theta_out[1] = t2 * scale;
    }
    __syncwarp();
}

// Residual test of the lowest Ritz pair of a cycle so far (steps 0..i).  With
// full reorthogonalisation the residual equals beta_i |s_m| (m = i + 1), s the
// lowest eigenvector of tridiag(alpha, beta) (Algorithm 2).  No eigenvector is
// formed: with p_k the characteristic polynomials of the leading k x k blocks
// (of T - x I), s_m^2 = -p_{m-1}(theta) / p_m'(theta).  theta comes from an FP32
// multisection and two FP64 Newton steps; at the last point x the first-order
// correction p_{m-1}(theta) ~ p_{m-1}(x) - (p_m(x) / p_m'(x)) p_{m-1}'(x)
// removes the error of x, so tiny |s_m| (a converged pair) are resolved.
// Returns, in every lane, whether beta_i |s_m| <= tol |theta|; a failed Newton
// step or a negative or non-finite s_m^2 counts as not converged.  One warp;
// work arrays as for tridiag_warp.
__device__ bool ritz_converged_warp(const double *alpha, const double *beta, int i, double tol, double *a,
                                    double *b, double *b2, double *z, double *u0, double *u1, double *u2)
{
    const int m = i + 1;
    const int lane = threadIdx.x & 31;
    const float scf = gershgorin_pow2(alpha, beta, m);
    const double inv = 1.0 / (double)scf;          // exact: a power of two
    float *af = reinterpret_cast<float *>(u0);
    float *b2f = reinterpret_cast<float *>(u1);
    for (int k = lane; k < m; k += 32) {
        a[k] = alpha[k] * inv;
        const double bk = (k + 1 < m) ? beta[k] * inv : 0.0;
        b2[k] = bk * bk;
        af[k] = (float)a[k];
        b2f[k] = (float)b2[k];
    }
    __syncwarp();
    float lo = -1.25f, hi = 1.25f;
    multisect<float>(af, b2f, m, 1, lo, hi, 4e-7f);
    __syncwarp();
    int ok = 0;
    if (lane == 0) {
        double x;
        CharPoly cp;
        if (newton_lowest(a, b2, m, lo, hi, 3, x, cp)) {
            const double rd = rcp64(cp.dpm);
            const double pm1 = cp.pm1 - cp.pm * rd * cp.dpm1;      // p_{m-1} at the refined eigenvalue
            const double s2 = -pm1 * rd;
            const double th = fabs(x - cp.pm * rd) * (double)scf;
            const double bi = beta[i];
            ok = s2 >= 0.0 && isfinite(s2) && isfinite(bi) && bi * bi * s2 <= (tol * th) * (tol * th);
        }
    }
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// After step i of a cycle: once its lowest Ritz pair meets tol the rest of
// the cycle is skipped (broken = 1); the restart from that Ritz vector follows
// at once, and its |beta_1/alpha_1| decides convergence as before.  One warp.
__global__ void ritz_estimate_kernel(LanczosScalars *S, int i, double tol)
{
    __shared__ double a[kMaxWindow], b[kMaxWindow], b2[kMaxWindow], z[kMaxWindow];
    __shared__ double u0[kMaxWindow], u1[kMaxWindow], u2[kMaxWindow];
    if (S->broken) return;                        // uniform: breakdown, or already converged
    const bool done = ritz_converged_warp(S->alpha, S->beta, i, tol, a, b, b2, z, u0, u1, u2);
    if (done && threadIdx.x == 0) S->broken = 1;
}

// Batched form: one warp per problem still running in the cycle
__global__ void batch_ritz_estimate_kernel(BatchState *S, int count, int i, double tol)
{
    __shared__ double work[4][7][kMaxWindow];
    const int wi = threadIdx.x >> 5;
    const int pr = blockIdx.x * 4 + wi;
    if (pr >= count) return;
    BatchState &P = S[pr];
    if (P.skip || P.used != i + 1) return;        // warp-uniform
    double (*w)[kMaxWindow] = work[wi];
    const bool done = ritz_converged_warp(P.alpha, P.beta, i, tol, w[0], w[1], w[2], w[3], w[4], w[5], w[6]);
    if (done && (threadIdx.x & 31) == 0) {
        P.broken = 1;
        P.skip = 1;
    }
}

__global__ void tridiag_kernel(LanczosScalars *S, int m)
{
    __shared__ double a[kMaxWindow], b[kMaxWindow], b2[kMaxWindow];
    __shared__ double z[kMaxWindow], u0[kMaxWindow], u1[kMaxWindow], u2[kMaxWindow];
    if (m <= 0) m = S->used;
    if (m < 1 || m > kMaxWindow) return;
    tridiag_warp(S->alpha, S->beta, m, S->theta, S->s, a, b, b2, z, u0, u1, u2);
}

// Q0 <- sum_j s_j Q_j for j < *m_dev (in place; each element is read by its own
// thread before that thread writes it), ||Q0||^2 partials
template <typename T, int W>
__global__ void __launch_bounds__(kThreads)
ritz_kernel(T *Q, int64_t ldq, const int *__restrict__ m_dev, const double *__restrict__ s, int64_t n,
            double *__restrict__ part, double *__restrict__ norm_out, unsigned long long *ticket)
{
    const int m = *m_dev;
    __shared__ T ss[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int j = threadIdx.x; j < m; j += kThreads) ss[j] = (T)s[j];
    __syncthreads();
    DotAcc<T> nrm;
    const int64_t nc = (n + W - 1) / W;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t e = (int64_t)blockIdx.x * kThreads + threadIdx.x; e < nc; e += stride) {
        Pack<T, W> v;
#pragma unroll
        for (int k = 0; k < W; ++k) v.v[k] = T(0);
        for (int j0 = 0; j0 < m; j0 += kGroup) {
            Pack<T, W> q[kGroup];
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m) q[u] = load_pack<T, W, false>(Q + (int64_t)(j0 + u) * ldq, e, n);
#pragma unroll
            for (int u = 0; u < kGroup; ++u)
                if (j0 + u < m)
#pragma unroll
                    for (int k = 0; k < W; ++k) v.v[k] = fma_t<T>(ss[j0 + u], q[u].v[k], v.v[k]);
        }
        store_pack<T, W>(Q, e, n, v);
#pragma unroll
        for (int k = 0; k < W; ++k) nrm.add(v.v[k], v.v[k]);
    }
    const double sum = block_reduce(nrm, sh);
    if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = sum;
    if (ticket && arrive_last(ticket)) reduce_partials(part, gridDim.x, 1, norm_out);
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

// r = a - lambda b (FP64), ||r||^2 partials; r stored when dst != nullptr
template <int W>
__global__ void __launch_bounds__(kThreads)
residual_kernel(const double *__restrict__ a, const double *__restrict__ b,
                const double *__restrict__ lambda, double *__restrict__ dst, int64_t n,
                double *__restrict__ part, double *__restrict__ norm_out, unsigned long long *ticket)
{
    __shared__ double sh[kThreads / 32];
    const double lam = *lambda;
    DotAcc<double> nrm;
    const int64_t nc = (n + W - 1) / W;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < nc; c += stride) {
        const Pack<double, W> x = load_pack<double, W, true>(a, c, n);
        const Pack<double, W> y = load_pack<double, W, true>(b, c, n);
        Pack<double, W> r;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            r.v[k] = x.v[k] - lam * y.v[k];
            nrm.add(r.v[k], r.v[k]);
        }
        if (dst) store_pack<double, W>(dst, c, n, r);
    }
    const double s = block_reduce(nrm, sh);
    if (threadIdx.x == 0) part[blockIdx.x * kMaxWindow] = s;
    if (ticket && arrive_last(ticket)) reduce_partials(part, gridDim.x, 1, norm_out);
}

// ---- batched (segmented) kernels: vectors concatenated over problems ---------
// Every chunk starts on a 16-byte boundary (problems and chunks are laid out on
// 4-element boundaries, and so is the stride between window vectors), so the
// kernels move 16-byte packs; the last pack of a chunk is read zero-filled and
// written element by element.
template <typename T>
__host__ __device__ constexpr int seg_w() { return kPackBytes / (int)sizeof(T); }

template <typename T>
__global__ void __launch_bounds__(kThreads)
seg_dots_kernel(const BatchVec V, const T *__restrict__ Q, int64_t ldq, int m, const T *__restrict__ v,
                const BatchState *__restrict__ S, int use_skip, double *__restrict__ part)
{
    constexpr int W = seg_w<T>();
    __shared__ double shg[kGroup * (kThreads / 32)];
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        if (use_skip && S[pr].skip) continue;                // CTA-uniform
        const int64_t e0 = V.chunk_start[c];
        const int len = V.chunk_len[c];
        const int np = (len + W - 1) / W;
        for (int j0 = 0; j0 < m; j0 += kGroup) {
            DotAcc<T> acc[kGroup];
            for (int e = threadIdx.x; e < np; e += kThreads) {
                const Pack<T, W> pv = load_pack<T, W, true>(v + e0, e, len);
                Pack<T, W> q[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq + e0, e, len);
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m)
#pragma unroll
                        for (int k = 0; k < W; ++k) acc[u].add(q[u].v[k], pv.v[k]);
            }
            block_reduce_group<T>(acc, min(kGroup, m - j0), shg, part + (int64_t)c * kMaxWindow + j0);
        }
    }
}

// one warp per (problem, output): lane l adds chunk l of the problem (<= 32 chunks).
// use_skip: 0 every problem, 1 pass over problems with skip set, 2 pass over done ones
__global__ void seg_reduce_kernel(const BatchVec V, int m, const BatchState *__restrict__ S, int use_skip,
                                  const double *__restrict__ part, double *__restrict__ out, int out_stride)
{
    const int w = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    const int pr = w / m, j = w - pr * m;
    if (pr >= V.count) return;
    if ((use_skip == 1 && S[pr].skip) || (use_skip == 2 && S[pr].done)) return;   // warp-uniform
    const int nc = V.prob_nchunk[pr], c0 = V.prob_chunk0[pr];
    double sum = lane < nc ? part[(int64_t)(c0 + lane) * kMaxWindow + j] : 0.0;
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) out[(int64_t)pr * out_stride + j] = sum;
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
seg_recur_project_kernel(const BatchVec V, const T *__restrict__ Q, int64_t ldq, int i, T *__restrict__ v,
                         const BatchState *__restrict__ S, double *__restrict__ part)
{
    constexpr int W = seg_w<T>();
    __shared__ double shg[kGroup * (kThreads / 32)];
    const int m = i + 1;
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        if (S[pr].skip) continue;
        const T a = (T)S[pr].c1;
        const T b = (T)(i > 0 ? S[pr].beta[i - 1] : 0.0);
        const int64_t e0 = V.chunk_start[c];
        const int len = V.chunk_len[c];
        const int np = (len + W - 1) / W;
        T *vc = v + e0;
        const T *qi = Q + (int64_t)i * ldq + e0;
        const T *qm = Q + (int64_t)(i > 0 ? i - 1 : 0) * ldq + e0;
        for (int j0 = 0; j0 < m; j0 += kGroup) {
            DotAcc<T> acc[kGroup];
            for (int e = threadIdx.x; e < np; e += kThreads) {
                Pack<T, W> x = load_pack<T, W, false>(vc, e, len);
                if (j0 == 0) {                                  // same thread, same pack in later groups
                    const Pack<T, W> yi = load_pack<T, W, true>(qi, e, len);
                    const Pack<T, W> ym = load_pack<T, W, true>(qm, e, len);
#pragma unroll
                    for (int k = 0; k < W; ++k) x.v[k] = fma_t<T>(-b, ym.v[k], fma_t<T>(-a, yi.v[k], x.v[k]));
                    store_pack<T, W>(vc, e, len, x);
                }
                Pack<T, W> q[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq + e0, e, len);
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m)
#pragma unroll
                        for (int k = 0; k < W; ++k) acc[u].add(q[u].v[k], x.v[k]);
            }
            block_reduce_group<T>(acc, min(kGroup, m - j0), shg, part + (int64_t)c * kMaxWindow + j0);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
seg_update_kernel(const BatchVec V, const T *__restrict__ Q, int64_t ldq, int m, T *__restrict__ v,
                  const BatchState *__restrict__ S, double *__restrict__ part)
{
    constexpr int W = seg_w<T>();
    __shared__ T sc[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        if (S[pr].skip) continue;
        __syncthreads();                                        // sc of the previous chunk consumed
        for (int j = threadIdx.x; j < m; j += kThreads) sc[j] = (T)S[pr].c2[j];
        __syncthreads();
        const int64_t e0 = V.chunk_start[c];
        const int len = V.chunk_len[c];
        const int np = (len + W - 1) / W;
        T *vc = v + e0;
        DotAcc<T> nrm;
        for (int e = threadIdx.x; e < np; e += kThreads) {
            Pack<T, W> x = load_pack<T, W, false>(vc, e, len);
            for (int j0 = 0; j0 < m; j0 += kGroup) {
                Pack<T, W> q[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m) q[u] = load_pack<T, W, true>(Q + (int64_t)(j0 + u) * ldq + e0, e, len);
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m)
#pragma unroll
                        for (int k = 0; k < W; ++k) x.v[k] = fma_t<T>(-sc[j0 + u], q[u].v[k], x.v[k]);
            }
            store_pack<T, W>(vc, e, len, x);
#pragma unroll
            for (int k = 0; k < W; ++k) nrm.add(x.v[k], x.v[k]);
        }
        const double sum = block_reduce(nrm, sh);
        if (threadIdx.x == 0) part[(int64_t)c * kMaxWindow] = sum;
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
seg_scale_kernel(const BatchVec V, const T *src, T *dst, const BatchState *__restrict__ S, int i, int mode)
{
    constexpr int W = seg_w<T>();
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        if (mode == 0 ? S[pr].skip : S[pr].done) continue;
        const double d = mode == 0 ? S[pr].beta[i] : sqrt(S[pr].norm2);
        const T f = (T)(d > 0.0 ? 1.0 / d : 0.0);
        const int64_t e0 = V.chunk_start[c];
        const int len = V.chunk_len[c];
        const int np = (len + W - 1) / W;
        for (int e = threadIdx.x; e < np; e += kThreads) {
            Pack<T, W> x = load_pack<T, W, false>(src + e0, e, len);
#pragma unroll
            for (int k = 0; k < W; ++k) x.v[k] = x.v[k] * f;
            store_pack<T, W>(dst + e0, e, len, x);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
seg_ritz_kernel(const BatchVec V, T *__restrict__ Q, int64_t ldq, const BatchState *__restrict__ S,
                double *__restrict__ part)
{
    constexpr int W = seg_w<T>();
    __shared__ T ss[kMaxWindow];
    __shared__ double sh[kThreads / 32];
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        if (S[pr].done) continue;
        const int m = S[pr].used;
        __syncthreads();
        for (int j = threadIdx.x; j < m; j += kThreads) ss[j] = (T)S[pr].s[j];
        __syncthreads();
        const int64_t e0 = V.chunk_start[c];
        const int len = V.chunk_len[c];
        const int np = (len + W - 1) / W;
        DotAcc<T> nrm;
        for (int e = threadIdx.x; e < np; e += kThreads) {
            Pack<T, W> x;
#pragma unroll
            for (int k = 0; k < W; ++k) x.v[k] = T(0);
            for (int j0 = 0; j0 < m; j0 += kGroup) {
                Pack<T, W> q[kGroup];
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m) q[u] = load_pack<T, W, false>(Q + (int64_t)(j0 + u) * ldq + e0, e, len);
#pragma unroll
                for (int u = 0; u < kGroup; ++u)
                    if (j0 + u < m)
#pragma unroll
                        for (int k = 0; k < W; ++k) x.v[k] = fma_t<T>(ss[j0 + u], q[u].v[k], x.v[k]);
            }
            store_pack<T, W>(Q + e0, e, len, x);              // Q_0, in place: this thread read it above
#pragma unroll
            for (int k = 0; k < W; ++k) nrm.add(x.v[k], x.v[k]);
        }
        const double sum = block_reduce(nrm, sh);
        if (threadIdx.x == 0) part[(int64_t)c * kMaxWindow] = sum;
    }
}

__global__ void __launch_bounds__(kThreads)
seg_residual_kernel(const BatchVec V, const double *__restrict__ w, const double *__restrict__ v,
                    const BatchState *__restrict__ S, double *__restrict__ part)
{
    __shared__ double sh[kThreads / 32];
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        const double lam = S[pr].e0;
        const int64_t e0 = V.chunk_start[c];
        const int len = V.chunk_len[c];
        double acc = 0.0;
        for (int e = threadIdx.x; e < len; e += kThreads) {
            const double r = w[e0 + e] - lam * v[e0 + e];
            acc = fma(r, r, acc);
        }
        const double sum = block_sum(acc, sh);
        if (threadIdx.x == 0) part[(int64_t)c * kMaxWindow] = sum;
    }
}

template <typename T>
__global__ void seg_random_kernel(const BatchVec V, T *__restrict__ q, uint64_t seed)
{
    for (int c = blockIdx.x; c < V.nchunks; c += gridDim.x) {
        const int pr = V.chunk_prob[c];
        const int64_t e0 = V.chunk_start[c];
        const int64_t local0 = e0 - V.prob_off[pr];
        const int len = V.chunk_len[c];
        for (int e = threadIdx.x; e < len; e += blockDim.x)
            q[e0 + e] = (T)splitmix_uniform(seed, (uint64_t)(local0 + e));
    }
}

__global__ void batch_reset_kernel(BatchState *S, int count)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= count) return;
    S[pr].used = 0;
    S[pr].broken = 0;
    S[pr].tnorm = 0.0;
    S[pr].skip = S[pr].done;
}

__global__ void batch_finalize_kernel(BatchState *S, int count, int i)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= count) return;
    BatchState &P = S[pr];
    if (P.skip) return;
    const double a = P.c1 + P.c2[i];
    const double b = sqrt(P.norm2);
    P.alpha[i] = a;
    P.beta[i] = b;
    const double tn = fmax(P.tnorm, fabs(a) + b + (i > 0 ? P.beta[i - 1] : 0.0));
    P.tnorm = tn;
    P.used = i + 1;
    P.iters += 1;
    if (!(b > 1e-13 * tn)) { P.broken = 1; P.skip = 1; }
}

__device__ __forceinline__ unsigned long long device_clock_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void batch_converge_kernel(BatchState *S, int count, double tol, const int *cycle_dev,
                                      int stall_check, int *active)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= count) return;
    BatchState &P = S[pr];
    if (P.done) return;
    const int cycle = *cycle_dev;
    const double a = P.alpha[0], b = P.beta[0];
    const double rel = (b == 0.0) ? 0.0 : b / fabs(a);
    P.rel = rel;
    P.e0 = a;
    bool stop = rel <= tol;
    if (!stop && stall_check) {
        const double old = P.hist[0];
        P.hist[0] = P.hist[1]; P.hist[1] = P.hist[2]; P.hist[2] = P.hist[3]; P.hist[3] = rel;
        if (cycle >= 3 && fp32_stalled(rel, old, tol)) { stop = true; P.stalled = 1; }
    }
    if (stop) {
        P.done = 1;
        P.skip = 1;
        P.done_cycle = cycle;
        P.t_done = device_clock_ns();
    } else {
        atomicAdd(active, 1);
    }
}

__global__ void batch_ctl_kernel(int *ctl, int max_cycles, cudaGraphConditionalHandle loop)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int active = ctl[0], cycle = ctl[1];
    cudaGraphSetConditional(loop, (active > 0 && cycle < max_cycles) ? 1u : 0u);
    ctl[1] = cycle + 1;
    ctl[0] = 0;
}

__global__ void device_clock_kernel(unsigned long long *t)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *t = device_clock_ns();
}

__global__ void batch_tridiag_kernel(BatchState *S, int count)
{
    __shared__ double work[4][7][kMaxWindow];
    const int wi = threadIdx.x >> 5;
    const int pr = blockIdx.x * 4 + wi;
    if (pr >= count) return;
    BatchState &P = S[pr];
    if (P.done || P.used < 1) return;                        // warp-uniform
    double (*w)[kMaxWindow] = work[wi];
    tridiag_warp(P.alpha, P.beta, P.used, P.theta, P.s, w[0], w[1], w[2], w[3], w[4], w[5], w[6]);
}

// after the FP64 refinement: problems whose residual misses tol are reopened
__global__ void batch_reopen_kernel(BatchState *S, int count, double tol, const int *next_cycle, int *reopened)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= count) return;
    BatchState &P = S[pr];
    if (P.rel <= tol) {                          // refined residual within tol: finished, the answer is final now
        if (!P.done) { P.done = 1; P.skip = 1; P.done_cycle = *next_cycle - 1; }
        P.t_done = device_clock_ns();
        return;
    }
    P.done = 0;
    P.skip = 0;
    P.stalled = 0;
    P.hist[0] = P.hist[1] = P.hist[2] = P.hist[3] = 0.0;
    atomicAdd(reopened, 1);
}

__global__ void batch_rayleigh_kernel(BatchState *S, int count, int stage)
{
    const int pr = blockIdx.x * blockDim.x + threadIdx.x;
    if (pr >= count) return;
    BatchState &P = S[pr];
    if (stage == 0) {
        P.e0 = P.c2[0] / P.c2[1];
    } else {
        const double r = sqrt(P.norm2 / P.c2[1]);
        P.rel = (r == 0.0) ? 0.0 : r / fabs(P.e0);
    }
}

int seg_grid(const BatchVec &V)
{
    const int cap = sm_count() * 8;
    int g = V.nchunks < cap ? V.nchunks : cap;
    return g > 0 ? g : 1;
}

inline int state_stride() { return (int)(sizeof(BatchState) / sizeof(double)); }

inline void seg_reduce(const BatchVec &V, int m, const BatchState *S, int use_skip, const double *part,
                       double *out, cudaStream_t st)
{
    const int64_t warps = (int64_t)V.count * m;
    const int blocks = (int)((warps * 32 + 255) / 256);
    seg_reduce_kernel<<<blocks, 256, 0, st>>>(V, m, S, use_skip, part, out, state_stride());
}

int grid_for(int64_t n)
{
    int64_t g = (n + kThreads - 1) / kThreads;
    if (g > grid_cap()) g = grid_cap();
    return (int)(g > 0 ? g : 1);
}

// 16-byte packs when every vector of the launch starts on a 16-byte boundary
// (and the leading dimension keeps it there); single elements otherwise
template <typename T>
bool packable(std::initializer_list<const void *> ptrs, int64_t ld)
{
    constexpr int W = kPackBytes / sizeof(T);
    if (ld % W) return false;
    for (const void *p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) % kPackBytes) return false;
    return true;
}

// CTAs of one wave of a streaming kernel: SMs x resident CTAs per SM (looked up
// once per kernel and device), at most grid_cap(), and no more than the work needs
template <auto kernel>
int wave_grid(int64_t units)
{
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        dev = 0;
    }
    int wave = cache[dev].load(std::memory_order_relaxed);
    if (wave <= 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess) {
            cudaGetLastError();
            per_sm = 1;
        }
        const int w = sm_count() * (per_sm > 0 ? per_sm : 1);
        wave = w < grid_cap() ? w : grid_cap();
        cache[dev].store(wave, std::memory_order_relaxed);
    }
    const int g = grid_for(units);
    return g < wave ? g : wave;
}

template <typename T>
int64_t pack_units(int64_t n, bool packed)
{
    constexpr int W = kPackBytes / sizeof(T);
    return packed ? (n + W - 1) / W : n;
}

template <typename T>
void dots_t(const T *Q, int64_t ld, int m, const T *p, int64_t n, double *part, double *out,
            unsigned long long *ticket, const int *skip, cudaStream_t st)
{
    constexpr int W = kPackBytes / sizeof(T);
    const bool pk = packable<T>({Q, p}, ld);
    const int g = pk ? wave_grid<dots_kernel<T, W>>(pack_units<T>(n, pk)) : wave_grid<dots_kernel<T, 1>>(n);
    if (m == 1) {
        if (pk) dots_kernel<T, W, 1><<<g, kThreads, 0, st>>>(Q, ld, m, p, n, part, out, ticket, skip);
        else dots_kernel<T, 1, 1><<<g, kThreads, 0, st>>>(Q, ld, m, p, n, part, out, ticket, skip);
    } else if (pk) {
        dots_kernel<T, W><<<g, kThreads, 0, st>>>(Q, ld, m, p, n, part, out, ticket, skip);
    } else {
        dots_kernel<T, 1><<<g, kThreads, 0, st>>>(Q, ld, m, p, n, part, out, ticket, skip);
    }
    count_launches(1);
    if (!ticket) reduce(part, g, m, out, st, skip);
}

template <typename T>
void recur_t(const T *Q, int64_t ld, int i, const LanczosScalars *S, T *p, int64_t n, double *part,
             double *out, unsigned long long *ticket, const int *skip, cudaStream_t st)
{
    constexpr int W = kPackBytes / sizeof(T);
    const bool pk = packable<T>({Q, p}, ld);
    const int g = pk ? wave_grid<recur_project_kernel<T, W>>(pack_units<T>(n, pk))
                     : wave_grid<recur_project_kernel<T, 1>>(n);
    if (pk) recur_project_kernel<T, W><<<g, kThreads, 0, st>>>(Q, ld, i, S, p, n, part, out, ticket, skip);
    else recur_project_kernel<T, 1><<<g, kThreads, 0, st>>>(Q, ld, i, S, p, n, part, out, ticket, skip);
    count_launches(1);
    if (!ticket) reduce(part, g, i + 1, out, st, skip);
}

template <typename T>
void update_t(const T *Q, int64_t ld, int m, const double *c, T *p, int64_t n, double *part, double *norm_out,
              unsigned long long *ticket, const int *skip, LanczosScalars *fin, int fin_i, cudaStream_t st)
{
    constexpr int W = kPackBytes / sizeof(T);
    const bool pk = packable<T>({Q, p}, ld);
    const int g = pk ? wave_grid<update_kernel<T, W>>(pack_units<T>(n, pk)) : wave_grid<update_kernel<T, 1>>(n);
    if (pk)
        update_kernel<T, W><<<g, kThreads, 0, st>>>(Q, ld, m, c, p, n, part, norm_out, ticket, skip, fin, fin_i);
    else
        update_kernel<T, 1><<<g, kThreads, 0, st>>>(Q, ld, m, c, p, n, part, norm_out, ticket, skip, fin, fin_i);
    count_launches(1);
    if (norm_out && !ticket) reduce(part, g, 1, norm_out, st, skip);
}

template <typename T>
void scale_t(const T *src, T *dst, int64_t n, const double *div, int is_norm2, const int *skip, cudaStream_t st)
{
    constexpr int W = kPackBytes / sizeof(T);
    const bool pk = packable<T>({src, dst}, 0);
    const int g = pk ? wave_grid<scale_kernel<T, W>>(pack_units<T>(n, pk)) : wave_grid<scale_kernel<T, 1>>(n);
    if (pk) scale_kernel<T, W><<<g, kThreads, 0, st>>>(src, dst, n, div, is_norm2, skip);
    else scale_kernel<T, 1><<<g, kThreads, 0, st>>>(src, dst, n, div, is_norm2, skip);
    count_launches(1);
}

template <typename T>
void ritz_t(T *Q, int64_t ld, const int *m_dev, const double *s, int64_t n, double *part, double *norm_out,
            unsigned long long *ticket, cudaStream_t st)
{
    constexpr int W = kPackBytes / sizeof(T);
    const bool pk = packable<T>({Q}, ld);
    const int g = pk ? wave_grid<ritz_kernel<T, W>>(pack_units<T>(n, pk)) : wave_grid<ritz_kernel<T, 1>>(n);
    if (pk) ritz_kernel<T, W><<<g, kThreads, 0, st>>>(Q, ld, m_dev, s, n, part, norm_out, ticket);
    else ritz_kernel<T, 1><<<g, kThreads, 0, st>>>(Q, ld, m_dev, s, n, part, norm_out, ticket);
    count_launches(1);
    if (!ticket) reduce(part, g, 1, norm_out, st);
}

// the step kernel instance of a plan and a group size
template <typename T, int KG>
const void *step_fn_kg(bool packed, bool in_smem)
{
    constexpr int W = kPackBytes / sizeof(T);
    if (packed)
        return in_smem ? (const void *)step_kernel<T, W, true, KG> : (const void *)step_kernel<T, W, false, KG>;
    return in_smem ? (const void *)step_kernel<T, 1, true, KG> : (const void *)step_kernel<T, 1, false, KG>;
}

template <typename T>
const void *step_fn(bool packed, bool in_smem, int kg)
{
    return kg <= 1   ? step_fn_kg<T, 1>(packed, in_smem)
           : kg <= 2 ? step_fn_kg<T, 2>(packed, in_smem)
           : kg <= 4 ? step_fn_kg<T, 4>(packed, in_smem)
                     : step_fn_kg<T, 8>(packed, in_smem);
}

// Group size for a step with m vectors in the window.  FP32: the fewest passes
// (8, or the power of two >= m).  FP64, whose multiply-adds occupy GB300's
// small FP64 pipe even when predicated off: the largest of 8, 4, 2, 1 whose
// last group leaves at most one vector slot idle.
template <typename T>
int step_group(int m)
{
    if (sizeof(T) == 4) return m >= 8 ? 8 : m > 2 ? 4 : m;
    for (int kg = 8; kg > 1; kg >>= 1)
        if ((kg - m % kg) % kg <= 1) return kg;
    return 1;
}

// the resident CTAs per SM of every group-size instance (the smallest)
template <typename T>
int step_per_sm(bool packed, bool in_smem, size_t smem)
{
    int lo = 1 << 30;
    for (int kg = 1; kg <= kGroup; kg <<= 1) {
        const void *fn = step_fn<T>(packed, in_smem, kg);
        if (in_smem && cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kStepThreads, in_smem ? smem : 0) !=
            cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        lo = std::min(lo, per_sm);
    }
    return lo;
}

template <typename T>
size_t step_pack_bytes(bool packed)
{
    return packed ? (size_t)kPackBytes : sizeof(T);
}

template <typename T>
int step_plan_t(int64_t n, int64_t ldq, const void *Q, const void *p, StepPlan *plan)
{
    plan->grid = 0;
    int dev = 0, coop = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) {
        cudaGetLastError();
        return 0;
    }
    const bool pk = packable<T>({Q, p}, ldq);
    const int64_t units = pack_units<T>(n, pk);
    const int64_t nchunk = (units + kStepThreads - 1) / kStepThreads;
    // at least four chunks of kStepThreads packs per CTA, at most one CTA per SM
    int64_t grid = std::min<int64_t>(std::max<int64_t>((nchunk + 3) / 4, 1), (int64_t)sm_count());
    int64_t slice = (nchunk + grid - 1) / grid * kStepThreads;      // packs per CTA, whole chunks
    const size_t smem = (size_t)slice * step_pack_bytes<T>(pk);
    bool in_smem = smem <= kStepSmemMax;
    int per_sm = in_smem ? step_per_sm<T>(pk, true, smem) : 0;
    if (per_sm < 1 || grid > (int64_t)per_sm * sm_count()) {   // without the slice in shared memory
        in_smem = false;
        per_sm = step_per_sm<T>(pk, false, 0);
        if (per_sm < 1) return 0;
        grid = std::min<int64_t>(grid, (int64_t)per_sm * sm_count());
        slice = (nchunk + grid - 1) / grid * kStepThreads;
    }
    plan->grid = (int)grid;
    plan->slice = slice;
    plan->packed = pk;
    plan->in_smem = in_smem;
    plan->smem = in_smem ? (size_t)slice * step_pack_bytes<T>(pk) : 0;
    return 1;
}

template <typename T>
cudaError_t step_t(const StepPlan &plan, const T *Q, int64_t ldq, int i, LanczosScalars *S, T *p, int64_t n,
                   double *part, GridBar *gb, T *qnext, cudaStream_t st)
{
    using P = typename StepRed<T>::P;
    P *pp = reinterpret_cast<P *>(part);
    void *args[] = {(void *)&Q, (void *)&ldq, (void *)&i, (void *)&S, (void *)&p, (void *)&n, (void *)&pp,
                    (void *)&gb, (void *)&qnext};
    const void *fn = step_fn<T>(plan.packed, plan.in_smem, step_group<T>(i + 1));
    const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(plan.grid), dim3(kStepThreads), args, plan.smem, st);
    count_launches(1);
    return e;
}

}  // namespace

int vec_grid() { return grid_cap(); }

int step_plan(int dtype, int64_t n, int64_t ldq, const void *Q, const void *p, StepPlan *plan)
{
    return dtype == 0 ? step_plan_t<double>(n, ldq, Q, p, plan) : step_plan_t<float>(n, ldq, Q, p, plan);
}

cudaError_t step_launch(int dtype, const StepPlan &plan, const void *Q, int64_t ldq, int i, LanczosScalars *S,
                        void *p, int64_t n, double *partials, GridBar *gb, void *qnext, cudaStream_t st)
{
    if (plan.grid < 1) return cudaErrorInvalidValue;
    if (dtype == 0)
        return step_t<double>(plan, (const double *)Q, ldq, i, S, (double *)p, n, partials, gb, (double *)qnext, st);
    return step_t<float>(plan, (const float *)Q, ldq, i, S, (float *)p, n, partials, gb, (float *)qnext, st);
}

cudaError_t multidot_launch(int dtype, const void *Q, int64_t ld, int m, const void *p, int64_t n,
                            double *partials, double *out, cudaStream_t st, const int *skip,
                            unsigned long long *ticket)
{
    if (dtype == 0) dots_t<double>((const double *)Q, ld, m, (const double *)p, n, partials, out, ticket, skip, st);
    else dots_t<float>((const float *)Q, ld, m, (const float *)p, n, partials, out, ticket, skip, st);
    return cudaGetLastError();
}

cudaError_t update_launch(int dtype, const void *Q, int64_t ld, int m, const double *c, void *p,
                          int64_t n, double *partials, double *norm_out, cudaStream_t st, const int *skip,
                          unsigned long long *ticket, LanczosScalars *fin, int fin_i)
{
    if (fin && (!norm_out || !ticket)) return cudaErrorInvalidValue;
    if (dtype == 0)
        update_t<double>((const double *)Q, ld, m, c, (double *)p, n, partials, norm_out, ticket, skip, fin, fin_i, st);
    else
        update_t<float>((const float *)Q, ld, m, c, (float *)p, n, partials, norm_out, ticket, skip, fin, fin_i, st);
    return cudaGetLastError();
}

cudaError_t scale_launch(int dtype, const void *src, void *dst, int64_t n, const double *div,
                         int div_is_norm2, cudaStream_t st, const int *skip)
{
    if (dtype == 0) scale_t<double>((const double *)src, (double *)dst, n, div, div_is_norm2, skip, st);
    else scale_t<float>((const float *)src, (float *)dst, n, div, div_is_norm2, skip, st);
    return cudaGetLastError();
}

cudaError_t recur_project_launch(int dtype, const void *Q, int64_t ld, int i, const LanczosScalars *S,
                                 void *p, int64_t n, double *partials, double *out, cudaStream_t st,
                                 const int *skip, unsigned long long *ticket)
{
    if (dtype == 0) recur_t<double>((const double *)Q, ld, i, S, (double *)p, n, partials, out, ticket, skip, st);
    else recur_t<float>((const float *)Q, ld, i, S, (float *)p, n, partials, out, ticket, skip, st);
    return cudaGetLastError();
}

cudaError_t quotient_launch(const double *num, const double *den, double *out, cudaStream_t st)
{
    quotient_kernel<<<1, 32, 0, st>>>(num, den, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t cycle_reset_launch(LanczosScalars *S, cudaStream_t st)
{
    cycle_reset_kernel<<<1, 32, 0, st>>>(S);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t ritz_estimate_launch(LanczosScalars *S, int i, double tol, cudaStream_t st)
{
    ritz_estimate_kernel<<<1, 32, 0, st>>>(S, i, tol);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_ritz_estimate_launch(BatchState *S, int count, int i, double tol, cudaStream_t st)
{
    batch_ritz_estimate_kernel<<<(count + 3) / 4, 128, 0, st>>>(S, count, i, tol);
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
                        double *partials, double *norm_out, cudaStream_t st, unsigned long long *ticket)
{
    if (dtype == 0) ritz_t<double>((double *)Q, ld, m_dev, s, n, partials, norm_out, ticket, st);
    else ritz_t<float>((float *)Q, ld, m_dev, s, n, partials, norm_out, ticket, st);
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
                            int64_t n, double *partials, double *norm_out, cudaStream_t st,
                            unsigned long long *ticket)
{
    const bool pk = packable<double>({a, b, dst}, 0);
    const int g = pk ? wave_grid<residual_kernel<2>>(pack_units<double>(n, pk)) : wave_grid<residual_kernel<1>>(n);
    if (pk) residual_kernel<2><<<g, kThreads, 0, st>>>(a, b, lambda, dst, n, partials, norm_out, ticket);
    else residual_kernel<1><<<g, kThreads, 0, st>>>(a, b, lambda, dst, n, partials, norm_out, ticket);
    count_launches(1);
    if (!ticket) reduce(partials, g, 1, norm_out, st);
    return cudaGetLastError();
}

// ---- batched launchers ---------------------------------------------------------
cudaError_t seg_dots_launch(int dtype, const BatchVec &V, const void *Q, int64_t ldq, int m, const void *v,
                            const BatchState *S, double *partials, double *out, int out_stride, cudaStream_t st)
{
    const int use_skip = S != nullptr;            // honour BatchState::skip
    const int g = seg_grid(V);
    if (dtype == 0)
        seg_dots_kernel<double><<<g, kThreads, 0, st>>>(V, (const double *)Q, ldq, m, (const double *)v, S, use_skip, partials);
    else
        seg_dots_kernel<float><<<g, kThreads, 0, st>>>(V, (const float *)Q, ldq, m, (const float *)v, S, use_skip, partials);
    const int64_t warps = (int64_t)V.count * m;
    seg_reduce_kernel<<<(int)((warps * 32 + 255) / 256), 256, 0, st>>>(V, m, S, use_skip, partials, out, out_stride);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t seg_recur_project_launch(int dtype, const BatchVec &V, const void *Q, int64_t ldq, int i, void *v,
                                     BatchState *S, double *partials, cudaStream_t st)
{
    const int g = seg_grid(V);
    if (dtype == 0)
        seg_recur_project_kernel<double><<<g, kThreads, 0, st>>>(V, (const double *)Q, ldq, i, (double *)v, S, partials);
    else
        seg_recur_project_kernel<float><<<g, kThreads, 0, st>>>(V, (const float *)Q, ldq, i, (float *)v, S, partials);
    seg_reduce(V, i + 1, S, 1, partials, &S[0].c2[0], st);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t seg_update_launch(int dtype, const BatchVec &V, const void *Q, int64_t ldq, int m, void *v,
                              BatchState *S, double *partials, cudaStream_t st)
{
    const int g = seg_grid(V);
    if (dtype == 0)
        seg_update_kernel<double><<<g, kThreads, 0, st>>>(V, (const double *)Q, ldq, m, (double *)v, S, partials);
    else
        seg_update_kernel<float><<<g, kThreads, 0, st>>>(V, (const float *)Q, ldq, m, (float *)v, S, partials);
    seg_reduce(V, 1, S, 1, partials, &S[0].norm2, st);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t seg_scale_launch(int dtype, const BatchVec &V, const void *src, void *dst, BatchState *S, int i,
                             int mode, cudaStream_t st)
{
    const int g = seg_grid(V);
    if (dtype == 0)
        seg_scale_kernel<double><<<g, kThreads, 0, st>>>(V, (const double *)src, (double *)dst, S, i, mode);
    else
        seg_scale_kernel<float><<<g, kThreads, 0, st>>>(V, (const float *)src, (float *)dst, S, i, mode);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t seg_ritz_launch(int dtype, const BatchVec &V, void *Q, int64_t ldq, BatchState *S, double *partials,
                            cudaStream_t st)
{
    const int g = seg_grid(V);
    if (dtype == 0)
        seg_ritz_kernel<double><<<g, kThreads, 0, st>>>(V, (double *)Q, ldq, S, partials);
    else
        seg_ritz_kernel<float><<<g, kThreads, 0, st>>>(V, (float *)Q, ldq, S, partials);
    seg_reduce(V, 1, S, 2, partials, &S[0].norm2, st);      // problems still running
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t seg_random_launch(int dtype, const BatchVec &V, void *q, uint64_t seed, cudaStream_t st)
{
    const int g = seg_grid(V);
    if (dtype == 0) seg_random_kernel<double><<<g, kThreads, 0, st>>>(V, (double *)q, seed);
    else seg_random_kernel<float><<<g, kThreads, 0, st>>>(V, (float *)q, seed);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t seg_residual_launch(const BatchVec &V, const double *w, const double *v, BatchState *S,
                                double *partials, cudaStream_t st)
{
    seg_residual_kernel<<<seg_grid(V), kThreads, 0, st>>>(V, w, v, S, partials);
    seg_reduce(V, 1, S, 0, partials, &S[0].norm2, st);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t batch_reset_launch(BatchState *S, int count, cudaStream_t st)
{
    batch_reset_kernel<<<(count + 127) / 128, 128, 0, st>>>(S, count);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_finalize_launch(BatchState *S, int count, int i, cudaStream_t st)
{
    batch_finalize_kernel<<<(count + 127) / 128, 128, 0, st>>>(S, count, i);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_converge_launch(BatchState *S, int count, double tol, const int *cycle, int stall_check,
                                  int *active, cudaStream_t st)
{
    batch_converge_kernel<<<(count + 127) / 128, 128, 0, st>>>(S, count, tol, cycle, stall_check, active);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_ctl_launch(int *ctl, int max_cycles, cudaGraphConditionalHandle loop, cudaStream_t st)
{
    batch_ctl_kernel<<<1, 32, 0, st>>>(ctl, max_cycles, loop);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t device_clock_launch(unsigned long long *t, cudaStream_t st)
{
    device_clock_kernel<<<1, 32, 0, st>>>(t);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_tridiag_launch(BatchState *S, int count, cudaStream_t st)
{
    batch_tridiag_kernel<<<(count + 3) / 4, 128, 0, st>>>(S, count);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_reopen_launch(BatchState *S, int count, double tol, const int *last_cycle, int *reopened,
                                cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(reopened, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    batch_reopen_kernel<<<(count + 127) / 128, 128, 0, st>>>(S, count, tol, last_cycle, reopened);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t batch_rayleigh_launch(BatchState *S, int count, int stage, cudaStream_t st)
{
    batch_rayleigh_kernel<<<(count + 127) / 128, 128, 0, st>>>(S, count, stage);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pd
