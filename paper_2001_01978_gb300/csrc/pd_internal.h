// pd_internal.h -- internal declarations shared by the CUDA translation units
// of libpairdiag (not part of the public ABI).
//
// Basis layout ("blocks").  The Omega orbits are split into L low orbits
// (0..L-1) and H = Omega - L high orbits.  A state s = (h << L) | l with k =
// popcount(l) low pairs and N - k high pairs.  In ascending integer order all
// states with the same high word h are contiguous, so the basis is a sequence
// of blocks, one per admissible high word, and
//     index(s) = base(h) + rank_L(l),
// where rank_L is the colex rank of l among L-bit words with k set bits and
// base(h) is the sum of C(L + p_j, ordinal_j) over the set bits of h (ordinals
// k+1..N).  Both parts are the paper's hash (Sec. 3.2) split at bit L.
#pragma once
struct pairdiag_mlp;
#include <atomic>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

namespace pd {

// ---- host helpers (pd_api.cu) ------------------------------------------------
// record a one-line error for pairdiag_last_error() and return `code`
int fail(int code, const char *fmt, ...);
// streaming multiprocessors of the current device (looked up once per device)
int sm_count();
constexpr int kMaxDevices = 64;      // device ordinals the per-device caches cover
uint64_t host_binom(int n, int m);                        // Pascal table, 0 outside 0 <= m <= n <= 63
uint64_t host_block_base(uint64_t hw, int L, int N);      // index of the block with high word hw
void words_with_popcount(int bits, int c, std::vector<uint64_t> &out);   // ascending

#define PD_CUDA(call)                                                                           \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return ::pd::fail(e_ == cudaErrorMemoryAllocation ? -2 : -5, "%s: %s (%s:%d)", #call, \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                      \
    } while (0)

#define PD_TRY(call)                \
    do {                            \
        int s_ = (call);            \
        if (s_ != 0) return s_;     \
    } while (0)

// kernels launched by the library (diagnostic counter, defined in pd_api.cu)
extern std::atomic<long long> g_kernel_launches;
inline void count_launches(int n) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

constexpr int kMaxOmega = 62;

// ---- device memory cache (pd_pool.cu) --------------------------------------
// pool_alloc: a cached block of the same rounded size, else cudaMalloc (the
// cache is emptied once and the call retried when the device is full).
// pool_free: the block returns to the cache; no queued work may still use it.
// Blocks not from the pool are passed to cudaFree.
cudaError_t pool_alloc(void **p, size_t bytes);
void pool_free(void *p);
size_t pool_cached_bytes();

// FP32 phase of the mixed form: stop giving cycles to FP32 vectors once the
// restart residual rel no longer falls.  old is its value three cycles
// earlier; FP32 stops when rel fell by less than 5 % over those cycles, or by
// less than 30 % within 20x of the FP32 target (the rounding floor of FP32
// vectors lies near that target).  A residual that falls slowly far above the
// target is slow convergence, which FP32 cycles serve as well as FP64 ones.
__host__ __device__ inline bool fp32_stalled(double rel, double old, double target)
{
    return rel > 0.95 * old || (rel < 20.0 * target && rel > 0.7 * old);
}
constexpr int kPackBytes = 16;       // streaming kernels move 16-byte packs of vector elements
constexpr int kMaxLow = 13;          // L <= 13: rank table of 2^L uint16 in shared memory
constexpr int kMaxWindow = 64;       // Lanczos vectors per cycle
constexpr int kBinomStride = 64;     // binom[n * 64 + m] = C(n, m)

struct Blocks {
    int omega, n, L, H;
    int64_t nblocks;
    int max_block;                   // max_k C(L, k) over admissible k
    int max_hh;                      // max over blocks of the number of high->high hops
    int max_stage;                   // max over blocks of the elements of all neighbour blocks
                                     // (ph C(L, k+1) + (H - ph) C(L, k-1))
    const uint64_t *blk_h;           // [nblocks] high words, ascending
    const uint64_t *blk_base;        // [nblocks] index of the block's first state
    const uint16_t *lowword;         // [2^L] L-bit words grouped by popcount, ascending
    const uint16_t *rankL;           // [2^L] rank of a word within its popcount group
    const uint64_t *binom;           // [64*64]
    int lo_off[kMaxLow + 2];         // group offsets into lowword
    int variant;                     // H*x kernel: 0 automatic, 1 staged per neighbour, 2 all staged
    // truncated model space (Sec. 3.5): kept_map[full index] = position among the
    // kept states, -1 for a dropped state; nullptr = the full space.  Vectors of
    // a truncated handle hold the kept states only, in basis order.
    const int32_t *kept_map;
    // the blocks holding at least one kept state (the truncated H*x walks only these)
    const uint64_t *kept_blk_h, *kept_blk_base;
    int64_t kept_nblocks;
};

// ---- many problems at once (batched solver) ---------------------------------
struct BatchDesc {                   // one problem of a batch (device array)
    int omega, n, L;                 // H = omega - L
    int g_off;                       // offset of its G in the concatenated G arrays
    int d_off;                       // offset of its d in the concatenated d arrays
    int tab_off;                     // offset of its L's tables in lowword_all / rankL_all
    int64_t vec_off;                 // offset of its first element in concatenated vectors
    int64_t dim;
};
struct BatchBlocks {
    int64_t nblocks;                 // all problems
    const uint32_t *blk_prob;        // [nblocks] owning problem, non-decreasing
    const uint64_t *blk_h;           // [nblocks] high word
    const uint64_t *blk_base;        // [nblocks] index of the block's first state within its problem
    const BatchDesc *desc;           // [count]
    const uint16_t *lowword_all;     // per-L tables, concatenated
    const uint16_t *rankL_all;
    const uint64_t *binom;
    int max_omega, max_L, max_H, max_block, max_hh;   // bounds for the shared-memory layout
    int max_n;                       // largest number of pairs
    int variant;                     // 1: neighbour blocks staged per hop class; 3: direct gathers
};

// Counters of a handle's kernels (device memory, zero when allocated).  Every
// kernel that uses a field leaves it at zero when it finishes: the CTA that
// arrives last resets it, so no memset is needed between launches.
struct GridBar {                     // grid-wide barrier of a cooperative launch
    unsigned int count;              // CTAs arrived at the current barrier
    unsigned int gen;                // generation: opened by the last CTA to arrive
    int err;                         // a wait gave up (the launch's results are void)
    int pad;
};
struct Tickets {
    unsigned long long hx_next;      // next block of a persistent H*x launch
    unsigned long long hx_done;      // CTAs of that launch that have finished
    unsigned long long vec_done;     // CTAs of a streaming kernel whose partial sums are written
    unsigned long long pad;
    GridBar bar;                     // the fused Lanczos step's barriers
};

#ifdef __CUDACC__
// ---- device reductions shared by the kernels ---------------------------------
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

// (ah, al) += (bh, bl) in float-float arithmetic (TwoSum, then renormalised)
__device__ __forceinline__ void ff_add(float &ah, float &al, float bh, float bl)
{
    const float s = ah + bh;
    const float z = s - ah;
    float e = (ah - (s - z)) + (bh - z);
    e += al + bl;
    const float h = s + e;
    al = e - (h - s);
    ah = h;
}

// warp-wide sum of one double per lane; result valid in lane 0
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// warp-wide float-float sum; result valid in lane 0
__device__ __forceinline__ void warp_sum_ff(float &hi, float &lo)
{
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_down_sync(0xffffffffu, hi, o);
        const float ol = __shfl_down_sync(0xffffffffu, lo, o);
        ff_add(hi, lo, oh, ol);
    }
}

// block-wide sum of one double per thread; result valid in thread 0.
// sh: at least blockDim.x / 32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double *sh)
{
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;
}

// block-wide float-float sum, converted to double once (thread 0 holds it):
// the whole reduction tree stays on the FP32 pipes.  sh: blockDim.x / 16 floats.
__device__ __forceinline__ double block_sum_ff(float hi, float lo, float *sh)
{
    warp_sum_ff(hi, lo);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) { sh[2 * w] = hi; sh[2 * w + 1] = lo; }
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        float th = 0.0f, tl = 0.0f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) ff_add(th, tl, sh[2 * i], sh[2 * i + 1]);
        r = (double)th + (double)tl;
    }
    return r;
}

// dot-product accumulator of a storage type: FP64 FMAs for double, float-float
// (exact products, TwoSum) for float
template <typename T>
struct DotAcc {
    double v = 0.0;
    __device__ __forceinline__ void add(T a, T b) { v = fma((double)a, (double)b, v); }
    __device__ __forceinline__ double get() const { return v; }
};
template <>
struct DotAcc<float> {
    float hi = 0.0f, lo = 0.0f;
    __device__ __forceinline__ void add(float a, float b) { ff_add_prod(hi, lo, a, b); }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};
// block-wide sum of the accumulators (thread 0); sh: blockDim.x / 32 doubles
__device__ __forceinline__ double block_reduce(const DotAcc<double> &a, double *sh) { return block_sum(a.get(), sh); }
__device__ __forceinline__ double block_reduce(const DotAcc<float> &a, double *sh)
{
    return block_sum_ff(a.hi, a.lo, reinterpret_cast<float *>(sh));
}
// warp-wide sum of the accumulators (lane 0)
__device__ __forceinline__ double warp_reduce(const DotAcc<double> &a) { return warp_sum(a.get()); }
__device__ __forceinline__ double warp_reduce(const DotAcc<float> &a)
{
    float hi = a.hi, lo = a.lo;
    warp_sum_ff(hi, lo);
    return (double)hi + (double)lo;
}

// Called by every thread of every CTA after thread 0 has written the CTA's
// partial sums.  Returns true in the one CTA that arrives last; by then the
// partial sums of all CTAs are visible to it (read them with __ldcg).  That CTA
// returns the ticket to zero.  No CTA waits for another.
__device__ __forceinline__ bool arrive_last(unsigned long long *ticket)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();                                       // release this CTA's partial sums
        const unsigned long long t = atomicAdd(ticket, 1ull);
        const int last = (t == (unsigned long long)gridDim.x - 1ull);
        if (last) {
            *ticket = 0ull;
            __threadfence();                                   // acquire the others'
        }
        s_last = last;
    }
    __syncthreads();
    return s_last != 0;
}

// out[j] = sum_b part[b * kMaxWindow + j] for j < m: warp w takes outputs w,
// w + warps, ...; each lane a fixed strided subset of b, then a fixed xor tree,
// so the order of the additions never changes.  Returns out[0] in thread 0.
__device__ __forceinline__ double reduce_partials(const double *part, int nb, int m, double *out)
{
    const int lane = threadIdx.x & 31, nw = (int)(blockDim.x >> 5);
    double first = 0.0;
    for (int j = (int)(threadIdx.x >> 5); j < m; j += nw) {
        double s = 0.0;
#pragma unroll 4
        for (int b = lane; b < nb; b += 32) s += __ldcg(part + (int64_t)b * kMaxWindow + j);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) out[j] = s;
        if (j == 0) first = s;
    }
    return first;
}
#endif  // __CUDACC__

// ---- H*x (pd_hx.cu) -------------------------------------------------------
// precision 0: double vectors / double accumulation with G64, d64
// precision 1: float vectors / float accumulation with G32, d32
// precision 2: float x (taken as exact), double y; float-float products and row
//              sums with Gff, dff (each value split as hi = fl(v), lo = fl(v - hi)):
//              FP64-accurate rows on the FP32 pipes (variant 3, full space only)
struct HxProblem {
    const double *G64, *d64;         // G [omega*omega], d_p = 2 e_p + G_pp
    const float *G32, *d32;
    const float2 *Gff, *dff;
};
// batched H*x: skip[p * skip_stride] != 0 passes over problem p (skip nullable).
// counter: two zeroed device counters (next block, finished CTAs); the last CTA
// returns both to zero, so no memset is needed between launches (graph-safe).
// precision 2 (float-float rows, x float, y double) runs the batched variant-3
// kernel whatever BB.variant says; hx_batch_grid(BB, 2) is 0 where it does not fit.
cudaError_t hx_batch_launch(const BatchBlocks &BB, const HxProblem &P, int precision, const void *x, void *y,
                            unsigned long long *counter, int grid, cudaStream_t st, const int *skip, int skip_stride);
int hx_batch_grid(const BatchBlocks &BB, int precision);
size_t hx_smem_bytes(const Blocks &B, int precision);
int hx_variant(const Blocks &B, int precision);   // kernel variant a launch will use (1 or 2)
// y = H x (Eq. 2 in the pair basis) over the persistent grid.
// skip (nullable, device): when *skip != 0 the launched kernels return at once.
// dot (nullable): also x^T y, the Lanczos alpha, with one partial sum per basis
// block in dot->blk_part[B.nblocks]; the last CTA adds them in block order into
// *dot->out (deterministic).
struct HxDot {
    double *blk_part;
    double *out;
};
cudaError_t hx_launch(const Blocks &B, const HxProblem &P, int precision, const void *x, void *y,
                      Tickets *tk, int grid, cudaStream_t st, const int *skip = nullptr,
                      const HxDot *dot = nullptr);
int hx_grid(const Blocks &B, int precision);
// Truncation (Sec. 3.5).  The bin of a state is floor((D - lo) / (hi - lo) * bins)
// in FP64, clamped to bins - 1, with D its diagonal element summed in ascending
// orbit order; lo/hi the extreme diagonal elements.
// hist (device, zeroed by the caller): counts of the bins b with
// lo_bin <= b < lo_bin + (nbuckets << shift), per bucket (b - lo_bin) >> shift
cudaError_t trunc_hist_launch(const Blocks &B, const double *d64, double lo, double hi, int64_t bins,
                              int64_t lo_bin, int shift, int nbuckets, unsigned long long *hist, int grid,
                              cudaStream_t st);
// blk_kept[b] = kept states of block b (bin <= cut)
cudaError_t trunc_count_launch(const Blocks &B, const double *d64, double lo, double hi, int64_t bins,
                               int64_t cut, int *blk_kept, int grid, cudaStream_t st);
// map[i] = blk_first[b] + rank among the kept states of its block, -1 if dropped
cudaError_t trunc_map_launch(const Blocks &B, const double *d64, double lo, double hi, int64_t bins,
                             int64_t cut, const int64_t *blk_first, int32_t *map, int grid, cudaStream_t st);
// Monopole_Min/Max/Posit_Min: partials[grid*3] scratch; out[0]=min, out[1]=max, out[2]=pos (as double bits)
cudaError_t monopole_launch(const Blocks &B, const double *d64, double *partials, int grid,
                            double *out, cudaStream_t st);
// occupation numbers: partial[grid*omega] scratch, out[omega]
cudaError_t occupations_launch(const Blocks &B, const double *v, double *partials, int grid,
                               double *out, cudaStream_t st);

// ---- basis (pd_basis.cu) --------------------------------------------------
cudaError_t basis_launch(int omega, int n, const uint64_t *binom, int64_t first, int64_t count,
                         uint64_t *out, cudaStream_t st);
cudaError_t rank_launch(int omega, int n, const uint64_t *binom, const uint64_t *states,
                        int64_t count, uint64_t *ranks, cudaStream_t st);

// ---- vector algebra and tridiagonal solve (pd_lanczos.cu) -------------------
struct LanczosScalars {              // lives in device memory
    double alpha[kMaxWindow];
    double beta[kMaxWindow];
    double c1[kMaxWindow];
    double c2[kMaxWindow];
    double s[kMaxWindow];
    double theta[2];
    double norm2;
    double dots[4];
    double tnorm;                    // running max_i |alpha_i| + beta_i + beta_{i-1}
    int    used;                     // valid Lanczos steps of the current cycle
    int    broken;                   // breakdown seen: later steps of the cycle are skipped
};
// CTAs of the streaming vector kernels on the current device: 4 per SM, at
// most kMaxVecGrid (the partial-sum buffers hold kMaxVecGrid rows)
constexpr int kMaxVecGrid = 1024;
int vec_grid();
// Streaming kernels: vectors of n elements; Q holds vectors j at Q + j*ld.  They
// move 16-byte packs when every vector is 16-byte aligned (ld a multiple of the
// pack), else single elements.  partials: [vec_grid() * kMaxWindow] doubles.
// ticket (nullable): with a ticket the last CTA adds the partial sums itself;
// without one a separate one-CTA reduction is launched.
cudaError_t multidot_launch(int dtype, const void *Q, int64_t ld, int m, const void *p, int64_t n,
                            double *partials, double *out, cudaStream_t st, const int *skip = nullptr,
                            unsigned long long *ticket = nullptr);
// p -= sum_j c[j] Q_j; if norm_out != nullptr also ||p||^2 -> *norm_out.
// fin (nullable, needs norm_out and ticket): the Lanczos step bookkeeping of
// step fin_i, done by the last CTA: alpha[i] = c1[0] + c2[i], beta[i] =
// sqrt(norm2), used = i + 1; broken is set when beta[i] <= 1e-13 * tnorm (an
// invariant subspace was found).
cudaError_t update_launch(int dtype, const void *Q, int64_t ld, int m, const double *c, void *p,
                          int64_t n, double *partials, double *norm_out, cudaStream_t st,
                          const int *skip = nullptr, unsigned long long *ticket = nullptr,
                          struct LanczosScalars *fin = nullptr, int fin_i = 0);
// dst = src * (1 / sqrt(*norm2)) (or src / *beta when is_norm == 0)
cudaError_t scale_launch(int dtype, const void *src, void *dst, int64_t n, const double *div,
                         int div_is_norm2, cudaStream_t st, const int *skip = nullptr);
// p <- p - S->c1[0] q_i - S->beta[i-1] q_{i-1} (Algorithm 2 recurrence), then
// out[j] = Q_j^T p for j <= i (the projections of one full Gram-Schmidt pass)
cudaError_t recur_project_launch(int dtype, const void *Q, int64_t ld, int i, const LanczosScalars *S,
                                 void *p, int64_t n, double *partials, double *out, cudaStream_t st,
                                 const int *skip = nullptr, unsigned long long *ticket = nullptr);
// One Lanczos step after the product p = H q_i (alpha = S->c1[0]) in a single
// cooperative launch: the recurrence, the projections c = Q^T p and
// p -= Q c of one full Gram-Schmidt pass, ||p||, the step bookkeeping of
// S (alpha_i, beta_i, tnorm, used, broken, c2) and, unless qnext is null or the
// step broke down, qnext = p / beta_i.  Grid-wide barriers in between; a wait
// that gives up sets gb->err.  step_plan returns 0 where no cooperative launch
// is possible (the caller then takes the three-kernel form).
struct StepPlan {
    int grid = 0;                    // CTAs (all resident)
    int64_t slice = 0;               // packs per CTA
    bool packed = false;             // 16-byte packs
    bool in_smem = false;            // each CTA keeps its slice of p in shared memory
    size_t smem = 0;                 // dynamic shared memory per CTA
};
constexpr size_t kStepSmemMax = 192 * 1024;
int step_plan(int dtype, int64_t n, int64_t ldq, const void *Q, const void *p, StepPlan *plan);
cudaError_t step_launch(int dtype, const StepPlan &plan, const void *Q, int64_t ldq, int i, LanczosScalars *S,
                        void *p, int64_t n, double *partials, GridBar *gb, void *qnext, cudaStream_t st);
// start of a cycle: used = 0, broken = 0, tnorm = 0
cudaError_t cycle_reset_launch(LanczosScalars *S, cudaStream_t st);
// *out = *num / *den (one thread)
cudaError_t quotient_launch(const double *num, const double *den, double *out, cudaStream_t st);
// after step i of a cycle: when the residual of the lowest Ritz pair of the
// steps so far is within tol of its Ritz value, set broken (the cycle ends)
cudaError_t ritz_estimate_launch(LanczosScalars *S, int i, double tol, cudaStream_t st);
// lowest two eigenvalues + lowest eigenvector of tridiag(alpha, beta) -> S->theta, S->s;
// size m, or S->used when m <= 0
cudaError_t tridiag_launch(LanczosScalars *S, int m, cudaStream_t st);
// Q0 = sum_j s_j Q_j (in place) for j < *m_dev, ||Q0||^2 -> *norm_out
cudaError_t ritz_launch(int dtype, void *Q, int64_t ld, const int *m_dev, const double *s, int64_t n,
                        double *partials, double *norm_out, cudaStream_t st,
                        unsigned long long *ticket = nullptr);
cudaError_t random_start_launch(int dtype, void *q, int64_t n, uint64_t seed, cudaStream_t st);
cudaError_t convert_launch(int dst_dtype, void *dst, int src_dtype, const void *src, int64_t n,
                           cudaStream_t st);
// dst = a - lambda * b (double), ||dst||^2 -> *norm_out; lambda read from device
cudaError_t residual_launch(const double *a, const double *b, const double *lambda, double *dst,
                            int64_t n, double *partials, double *norm_out, cudaStream_t st,
                            unsigned long long *ticket = nullptr);

// ---- batched Lanczos (pd_lanczos.cu kernels, pd_batch.cu driver) -------------
struct BatchState {                  // one problem (device memory)
    double alpha[kMaxWindow];
    double beta[kMaxWindow];
    double c2[kMaxWindow];           // projections; also refinement scratch
    double s[kMaxWindow];            // ground Ritz vector of the cycle's L matrix
    double c1;                       // alpha from the three-term recurrence
    double norm2, tnorm;
    double theta[2];
    double e0, rel;                  // energy estimate and |beta_1/alpha_1| (or FP64 residual)
    double hist[4];                  // last restart residuals (stagnation test)
    int used, broken, done, skip;    // skip = done || broken (kernels pass over the problem)
    int iters, done_cycle, stalled, pad;
    unsigned long long t_done;       // device clock (ns) when the problem's answer was final
};
struct BatchVec {                    // vectors concatenated over problems, cut into chunks
    int count;
    int nchunks;                     // every chunk lies inside one problem; <= 32 per problem
    int64_t total;                   // elements per vector: every problem starts on a 4-element
                                     // boundary, and so does every chunk (up to 3 unused
                                     // elements after each problem)
    const int *chunk_prob;
    const int64_t *chunk_start;      // global element index
    const int *chunk_len;
    const int *prob_chunk0;          // [count] first chunk of each problem
    const int *prob_nchunk;          // [count]
    const int64_t *prob_off;         // [count] first element of each problem
};
constexpr int kMaxChunksPerProblem = 32;

// out[p * out_stride + j] = sum over problem p's elements of Q_j[e] v[e], j < m
// (Q vector-major with leading dimension ldq); skipped problems are left alone
// S (nullable): the problems' states; when given, problems with skip set are passed over
cudaError_t seg_dots_launch(int dtype, const BatchVec &V, const void *Q, int64_t ldq, int m, const void *v,
                            const BatchState *S, double *partials, double *out, int out_stride, cudaStream_t st);
// per problem: v <- v - c1 q_i - beta[i-1] q_{i-1}; then c2[j] = Q_j^T v, j <= i
cudaError_t seg_recur_project_launch(int dtype, const BatchVec &V, const void *Q, int64_t ldq, int i, void *v,
                                     BatchState *S, double *partials, cudaStream_t st);
// per problem: v <- v - sum_{j<m} c2[j] Q_j, norm2 = ||v||^2
cudaError_t seg_update_launch(int dtype, const BatchVec &V, const void *Q, int64_t ldq, int m, void *v,
                              BatchState *S, double *partials, cudaStream_t st);
// dst <- src / beta[i] (mode 0) or src / sqrt(norm2) (mode 1), per problem
cudaError_t seg_scale_launch(int dtype, const BatchVec &V, const void *src, void *dst, BatchState *S, int i,
                             int mode, cudaStream_t st);
// Q_0 <- sum_{j<used} s[j] Q_j per problem, norm2 = ||Q_0||^2
cudaError_t seg_ritz_launch(int dtype, const BatchVec &V, void *Q, int64_t ldq, BatchState *S, double *partials,
                            cudaStream_t st);
cudaError_t seg_random_launch(int dtype, const BatchVec &V, void *q, uint64_t seed, cudaStream_t st);
// per problem: residual r = w - e0 v (FP64), norm2 = ||r||^2
cudaError_t seg_residual_launch(const BatchVec &V, const double *w, const double *v, BatchState *S,
                                double *partials, cudaStream_t st);
cudaError_t batch_reset_launch(BatchState *S, int count, cudaStream_t st);
cudaError_t batch_finalize_launch(BatchState *S, int count, int i, cudaStream_t st);
// after step 0 of a cycle: convergence / stagnation per problem; *active += problems
// still running; the cycle number is read from *cycle (device)
cudaError_t batch_converge_launch(BatchState *S, int count, double tol, const int *cycle, int stall_check,
                                  int *active, cudaStream_t st);
// end of a cycle's convergence test, one thread: the device-side loop condition
// (problems still running and cycles left), then ctl[1] += 1 and ctl[0] = 0.
// ctl[0] = running problems, ctl[1] = cycle number.
cudaError_t batch_ctl_launch(int *ctl, int max_cycles, cudaGraphConditionalHandle loop, cudaStream_t st);
// *t = the device clock in ns
cudaError_t device_clock_launch(unsigned long long *t, cudaStream_t st);
cudaError_t batch_tridiag_launch(BatchState *S, int count, cudaStream_t st);
// after refinement: problems with rel > tol reopen (done = skip = 0), the others are
// finished; *reopened = number reopened
cudaError_t batch_reopen_launch(BatchState *S, int count, double tol, const int *last_cycle, int *reopened,
                                cudaStream_t st);
// e0 = c2[0] / c2[1] (Rayleigh quotient from v^T w and v^T v)
cudaError_t batch_rayleigh_launch(BatchState *S, int count, int stage, cudaStream_t st);

// ---- learned warm start (pd_mlp.cu) ----------------------------------------------
void mlp_features(int omega, int n, const double *e, const double *G, float *X);   // [omega x 16]
// start vector v[s] = exp(sum_{p in s} w_p - max) on storage type dtype (synchronous)
// scratch: 2^L device doubles (nullable); asynchronous on st
int product_start(const Blocks &B, const double *w_host, int dtype, void *v, cudaStream_t st,
                  double *scratch = nullptr);
// weighted least-squares per-orbit weights of a normalised FP64 vector (synchronous)
int product_fit(const Blocks &B, const double *v, double *w_out, cudaStream_t st);
int mlp_predict(struct ::pairdiag_mlp *m, int omega, int n, const double *e, const double *G, double *w_out);
// product start vectors of every problem of a batch from one network pass (synchronous)
int batch_mlp_start(struct ::pairdiag_mlp *m, const BatchBlocks &BB, int count, const int *omega, const int *n_pairs,
                    const double *e_all, const double *G_all, int dtype, void *v, cudaStream_t st);

}  // namespace pd
