// pd_basis.cu -- basis enumeration and ranking through the combinatorial
// number system (Sec. 3.1 basis in ascending order; Sec. 3.2 hash).
//
// The paper generates the basis serially with the '01' inversion successor
// (Algorithm 1).  On the GPU every index is independent: state(r) is the
// colex unranking of r (the largest orbit p_N with C(p_N, N) <= r, then the
// next one for the remainder, ...), so each thread writes its own word and
// the output is coalesced.  rank(s) = sum_j C(p_j, j) over the set bits of s
// in ascending order, which is the paper's hash minus one.
#include "pd_internal.h"

namespace pd {
namespace {

__global__ void basis_kernel(int omega, int n, const uint64_t *__restrict__ binom, int64_t first,
                             int64_t count, uint64_t *__restrict__ out)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count;
         idx += (int64_t)gridDim.x * blockDim.x) {
        uint64_t r = (uint64_t)(first + idx);
        uint64_t s = 0;
        int p = omega - 1;
        for (int i = n; i >= 1; --i) {
            uint64_t c;
            while ((c = __ldg(binom + p * kBinomStride + i)) > r) --p;
            s |= 1ull << p;
            r -= c;
            --p;
        }
        out[idx] = s;
    }
}

__global__ void rank_kernel(int omega, int n, const uint64_t *__restrict__ binom,
                            const uint64_t *__restrict__ states, int64_t count,
                            uint64_t *__restrict__ ranks)
{
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < count;
         idx += (int64_t)gridDim.x * blockDim.x) {
        uint64_t s = states[idx];
        const bool ok = __popcll(s) == n && (omega == 64 || (s >> omega) == 0);
        uint64_t r = 0;
        int ord = 0;
        while (s) {
            const int p = __ffsll((long long)s) - 1;
            s &= s - 1;
            ++ord;
            r += __ldg(binom + p * kBinomStride + ord);
        }
        ranks[idx] = ok ? r : ~0ull;
    }
}

int grid_for(int64_t count)
{
    int64_t g = (count + 255) / 256;
    if (g > sm_count() * 32) g = sm_count() * 32;
    return (int)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t basis_launch(int omega, int n, const uint64_t *binom, int64_t first, int64_t count,
                         uint64_t *out, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    basis_kernel<<<grid_for(count), 256, 0, st>>>(omega, n, binom, first, count, out);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t rank_launch(int omega, int n, const uint64_t *binom, const uint64_t *states,
                        int64_t count, uint64_t *ranks, cudaStream_t st)
{
    if (count <= 0) return cudaSuccess;
    rank_kernel<<<grid_for(count), 256, 0, st>>>(omega, n, binom, states, count, ranks);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pd
