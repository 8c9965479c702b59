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
#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

namespace pd {

// kernels launched by the library (diagnostic counter, defined in pd_api.cu)
extern std::atomic<long long> g_kernel_launches;
inline void count_launches(int n) { g_kernel_launches.fetch_add(n, std::memory_order_relaxed); }

constexpr int kMaxOmega = 62;
constexpr int kMaxLow = 13;          // L <= 13: rank table of 2^L uint16 in shared memory
constexpr int kMaxWindow = 64;       // Lanczos vectors per cycle
constexpr int kBinomStride = 64;     // binom[n * 64 + m] = C(n, m)

struct Blocks {
    int omega, n, L, H;
    int64_t nblocks;
    int max_block;                   // max_k C(L, k) over admissible k
    int max_hh;                      // max over blocks of the number of high->high hops
    const uint64_t *blk_h;           // [nblocks] high words, ascending
    const uint64_t *blk_base;        // [nblocks] index of the block's first state
    const uint16_t *lowword;         // [2^L] L-bit words grouped by popcount, ascending
    const uint16_t *rankL;           // [2^L] rank of a word within its popcount group
    const uint64_t *binom;           // [64*64]
    int lo_off[kMaxLow + 2];         // group offsets into lowword
    int variant;                     // H*x kernel: 0 automatic, 1 staged per neighbour, 2 all staged
};

// ---- H*x (pd_hx.cu) -------------------------------------------------------
// precision 0: double vectors / double accumulation with G64, d64
// precision 1: float vectors / float accumulation with G32, d32
struct HxProblem {
    const double *G64, *d64;         // G [omega*omega], d_p = 2 e_p + G_pp
    const float *G32, *d32;
};
size_t hx_smem_bytes(const Blocks &B, int precision);
int hx_variant(const Blocks &B, int precision);   // kernel variant a launch will use (1 or 2)
// skip (nullable, device): when *skip != 0 the launched kernels return at once
cudaError_t hx_launch(const Blocks &B, const HxProblem &P, int precision, const void *x, void *y,
                      int *counter, int grid, cudaStream_t st, const int *skip = nullptr);
int hx_grid(const Blocks &B, int precision);
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
int vec_grid();                      // CTAs of the streaming vector kernels
// partial results of the streaming kernels: [vec_grid() * kMaxWindow] doubles
cudaError_t multidot_launch(int dtype, const void *Q, int64_t ld, int m, const void *p, int64_t n,
                            double *partials, double *out, cudaStream_t st, const int *skip = nullptr);
// p -= sum_j c[j] Q_j; if norm_out != nullptr also ||p||^2 -> *norm_out
cudaError_t update_launch(int dtype, const void *Q, int64_t ld, int m, const double *c, void *p,
                          int64_t n, double *partials, double *norm_out, cudaStream_t st,
                          const int *skip = nullptr);
// dst = src * (1 / sqrt(*norm2)) (or src / *beta when is_norm == 0)
cudaError_t scale_launch(int dtype, const void *src, void *dst, int64_t n, const double *div,
                         int div_is_norm2, cudaStream_t st, const int *skip = nullptr);
// p <- p - S->c1[0] q_i - S->beta[i-1] q_{i-1} (Algorithm 2 recurrence), then
// out[j] = Q_j^T p for j <= i (the projections of one full Gram-Schmidt pass)
cudaError_t recur_project_launch(int dtype, const void *Q, int64_t ld, int i, const LanczosScalars *S,
                                 void *p, int64_t n, double *partials, double *out, cudaStream_t st,
                                 const int *skip = nullptr);
// Lanczos step bookkeeping: alpha[i] = c1[0]+c2[i], beta[i] = sqrt(norm2), used = i+1;
// sets broken when beta[i] <= 1e-13 * tnorm (an invariant subspace was found)
cudaError_t finalize_step_launch(LanczosScalars *S, int i, cudaStream_t st);
// start of a cycle: used = 0, broken = 0, tnorm = 0
cudaError_t cycle_reset_launch(LanczosScalars *S, cudaStream_t st);
// lowest two eigenvalues + lowest eigenvector of tridiag(alpha, beta) -> S->theta, S->s;
// size m, or S->used when m <= 0
cudaError_t tridiag_launch(LanczosScalars *S, int m, cudaStream_t st);
// Q0 = sum_j s_j Q_j (in place) for j < *m_dev, ||Q0||^2 -> *norm_out
cudaError_t ritz_launch(int dtype, void *Q, int64_t ld, const int *m_dev, const double *s, int64_t n,
                        double *partials, double *norm_out, cudaStream_t st);
cudaError_t random_start_launch(int dtype, void *q, int64_t n, uint64_t seed, cudaStream_t st);
cudaError_t convert_launch(int dst_dtype, void *dst, int src_dtype, const void *src, int64_t n,
                           cudaStream_t st);
// dst = a - lambda * b (double), ||dst||^2 -> *norm_out; lambda read from device
cudaError_t residual_launch(const double *a, const double *b, const double *lambda, double *dst,
                            int64_t n, double *partials, double *norm_out, cudaStream_t st);

}  // namespace pd
