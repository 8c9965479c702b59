// pd_hx.cu -- on-the-fly H*x in the seniority-zero pair basis (Sec. 3.3 and
// Eq. "diagonal" of the paper), plus the per-row reductions that share its
// block structure (Monopole_Min/Max, occupation numbers).
//
// y_s = (sum_{p in s} d_p) x_s + sum_{o in s, e not in s} G_eo x_{t(s,o,e)},
// d_p = 2 e_p + G_pp, t = s with the pair moved from orbit o to orbit e.
//
// One CTA owns one basis block at a time (all states sharing a high word h,
// see pd_internal.h); blocks are handed out through an atomic counter so that
// blocks of different sizes balance across the persistent grid.  For the
// block's rows (low words l, one or more per thread) the N(Omega-N) hops fall
// into four classes:
//   low->low   : target in the same block; x block staged in shared memory,
//                target offset from the shared rank table of L-bit words;
//   high->high : target block h^o^e has the SAME row offsets, so the gather is
//                a contiguous, coalesced read of that block with one
//                CTA-uniform coefficient G_eo;
//   high->low  : target block h - o (k+1 low pairs) staged in shared memory
//                once and reused by all rows and all empty low orbits;
//   low->high  : target block h + e (k-1 low pairs), likewise.
// No tensor cores: this is a sparse gather, not a dense contraction.
#include "pd_internal.h"

#include <cstdio>
#include <type_traits>

namespace pd {
namespace {

constexpr int kThreads = 256;

template <typename A>
struct HHop {            // one high->high hop of the current block
    uint64_t base;       // first index of the target block
    A g;                 // G_eo
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

struct Layout {
    size_t G, d, rank, x, xn, hh, mx, total;
};

template <typename T, typename A>
__host__ __device__ inline Layout layout(int omega, int L, int H, int max_block, int max_hh)
{
    Layout s;
    size_t off = 0;
    s.G = off;    off = align16(off + sizeof(A) * omega * omega);
    s.d = off;    off = align16(off + sizeof(A) * omega);
    s.rank = off; off = align16(off + sizeof(uint16_t) * (size_t(1) << L));
    s.x = off;    off = align16(off + sizeof(T) * max_block);
    s.xn = off;   off = align16(off + sizeof(T) * max_block);
    s.hh = off;   off = align16(off + sizeof(HHop<A>) * (max_hh > 0 ? max_hh : 1));
    s.mx = off;   off = align16(off + sizeof(uint64_t) * (H > 0 ? H : 1));
    s.total = off;
    return s;
}

// position of the n-th (0-based) set bit of w
__device__ __forceinline__ int nth_set_bit(uint64_t w, int n)
{
    for (int i = 0; i < n; ++i) w &= w - 1;
    return __ffsll((long long)w) - 1;
}

// index of the first state of the block with high word h (Sec. 3.2 hash,
// restricted to the high bits: ordinals k+1..N at positions L+p)
__device__ __forceinline__ uint64_t block_base(uint64_t h, int L, int N,
                                               const uint64_t *__restrict__ binom)
{
    int ord = N - __popcll(h);
    uint64_t s = 0;
    while (h) {
        const int p = __ffsll((long long)h) - 1;
        h &= h - 1;
        ++ord;
        s += __ldg(binom + (L + p) * kBinomStride + ord);
    }
    return s;
}

// x at full index i of a truncated space: the kept state's element, 0 for a
// dropped state (a hop to it contributes nothing: the principal submatrix)
template <typename T>
__device__ __forceinline__ T x_kept(const T *__restrict__ x, const int32_t *__restrict__ map, uint64_t i)
{
    const int32_t m = __ldg(map + i);
    return m >= 0 ? __ldg(x + m) : T(0);
}

// Float-float number hi + lo: the row sums of the FP64-accurate product of an
// FP32 vector, on the FP32 pipes (GB300 issues FP32 FMAs at 64 times its FP64
// rate).  A coefficient c is stored split, hi = fl(c), lo = fl(c - hi); its
// product with a vector element x, an FP32 value, is hi*x exactly (the
// rounding error recovered with one FMA) plus lo*x rounded once, so a product
// carries a relative error near 2^-48.  Sums add the high parts with Knuth's
// TwoSum and collect the low parts and the TwoSum errors in lo.
struct FF {
    float hi, lo;
    FF() = default;
    __host__ __device__ FF(float x) : hi(x), lo(0.0f) {}
    __host__ __device__ FF(float h, float l) : hi(h), lo(l) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ explicit operator float() const { return hi + lo; }
};
// a coefficient times a vector element (the element's lo is 0)
__device__ __forceinline__ FF operator*(FF c, FF x)
{
    const float p = c.hi * x.hi;
    return FF(p, fmaf(c.lo, x.hi, fmaf(c.hi, x.hi, -p)));
}
__device__ __forceinline__ FF &operator+=(FF &a, FF b)
{
    const float s = a.hi + b.hi;
    const float z = s - a.hi;
    const float t = (a.hi - (s - z)) + (b.hi - z);
    a.lo += b.lo + t;
    a.hi = s;
    return a;
}
__device__ __forceinline__ FF operator+(FF a, FF b)
{
    a += b;
    return a;
}

// x^T y over this warp's rows of one basis block (y as stored) into sw[warp]
// (lane 0).  No barrier: thread 0 adds the warp sums in warp order after the
// barrier that opens the next block (block_sum_deferred).
template <typename T, typename A, int R>
__device__ __forceinline__ void warp_dot(const A *acc, const T *sx, int nk, double *sw)
{
    // float-float rows: the dot in FP64 of the rows as written (FP64)
    using D = typename std::conditional<std::is_same<A, FF>::value, double, T>::type;
    DotAcc<D> d;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = threadIdx.x + i * kThreads;
        if (r < nk) d.add((D)sx[r], D(acc[i]));
    }
    const double s = warp_reduce(d);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
}

// Thread 0, after a barrier: the previous block's warp sums into blk_part[prev]
__device__ __forceinline__ void block_sum_deferred(double *blk_part, long long prev, const double *sw)
{
    if (!blk_part || prev < 0) return;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += sw[w];
    blk_part[prev] = s;
}

// End of a persistent H*x launch, called by every CTA: the last one to arrive
// returns the work counter to zero and adds the per-block dot products in
// block order (a fixed order, so alpha does not depend on the schedule).
__device__ __forceinline__ void hx_finish(Tickets *tk, int64_t nblocks, const double *blk_part, double *dot_out,
                                          double *sred)
{
    if (!arrive_last(&tk->hx_done)) return;
    if (threadIdx.x == 0) tk->hx_next = 0ull;
    if (!blk_part) return;
    double s = 0.0;
#pragma unroll 8
    for (int64_t b = threadIdx.x; b < nblocks; b += blockDim.x) s += __ldcg(blk_part + b);
    s = block_sum(s, sred);
    if (threadIdx.x == 0) *dot_out = s;
}

// One basis block (high word h, first index base) of y = H x.  x and y point at
// the problem's own vector; sG/sd/sRank hold its G, d and rank table.  Called
// by every thread of the CTA (it contains barriers).  swdot (nullable): the
// block's x^T y per warp (warp_dot).
template <typename T, typename A, int R, bool TR = false>
__device__ __forceinline__ void hx_block(const int omega, const int L, const int H, const int N,
                                         const uint64_t h, const uint64_t base,
                                         const uint16_t *__restrict__ lowword,
                                         const uint64_t *__restrict__ binom,
                                         const A *sG, const A *sd, const uint16_t *sRank, T *sx, T *sxn,
                                         HHop<A> *sHH, uint64_t *sMX, const T *__restrict__ x,
                                         T *__restrict__ y, double *swdot,
                                         const int32_t *__restrict__ map = nullptr)
{
    const int tid = threadIdx.x;
    const uint32_t maskL = (1u << L) - 1u;
    const uint64_t maskH = (H >= 64) ? ~0ull : ((1ull << H) - 1ull);
    const int ph = __popcll(h);
    const int k = N - ph;                     // pairs in the low orbits
    const int nk = (int)__ldg(binom + L * kBinomStride + k);
    int lo_off_k = 0;
    for (int j = 0; j < k; ++j) lo_off_k += (int)__ldg(binom + L * kBinomStride + j);
    const uint16_t *lw = lowword + lo_off_k;
    const int nemp = H - ph;
    const int nhh = ph * nemp;

    // CTA-uniform hop tables of this block
    for (int t = tid; t < nhh; t += kThreads) {
        const int a = t / nemp, c = t - a * nemp;
        const int o = nth_set_bit(h, a);
        const int q = nth_set_bit(~h & maskH, c);
        sHH[t].base = block_base(h ^ (1ull << o) ^ (1ull << q), L, N, binom);
        sHH[t].g = sG[(L + q) * omega + (L + o)];
    }
    for (int t = tid; t < H; t += kThreads) {
        const uint64_t bit = 1ull << t;
        const bool occ = (h & bit) != 0;
        const bool ok = occ ? (k + 1 <= L) : (k >= 1);
        sMX[t] = ok ? block_base(h ^ bit, L, N, binom) : ~0ull;
    }
    for (int r = tid; r < nk; r += kThreads) sx[r] = TR ? x_kept(x, map, base + r) : x[base + r];
    __syncthreads();

    A Dh = A(0);
    for (uint64_t w = h; w; w &= w - 1) Dh += sd[L + __ffsll((long long)w) - 1];

    uint32_t lr[R];
    A acc[R];
    bool act[R];                              // rows of this thread that are computed (kept, if truncated)
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * kThreads;
        lr[i] = 0;
        acc[i] = A(0);
        act[i] = r < nk && (!TR || __ldg(map + base + r) >= 0);
        if (act[i]) {
            const uint32_t l = lw[r];
            lr[i] = l;
            A D = A(0);
            for (uint32_t w = l; w; w &= w - 1) D += sd[__ffs(w) - 1];
            acc[i] = (D + Dh) * A(sx[r]);
        }
    }

    // low -> low
    if (k > 0 && k < L) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (act[i]) {
                const uint32_t l = lr[i];
                A a = acc[i];
                uint32_t occ = l;
                for (int u = 0; u < k; ++u) {
                    const int o = __ffs(occ) - 1;
                    occ &= occ - 1;
                    const uint32_t lo = l ^ (1u << o);
                    uint32_t emp = ~l & maskL;
                    for (int v = 0; v < L - k; ++v) {
                        const int q = __ffs(emp) - 1;
                        emp &= emp - 1;
                        a += sG[q * omega + o] * A(sx[sRank[lo | (1u << q)]]);
                    }
                }
                acc[i] = a;
            }
        }
    }

    // high -> high: same offsets in the target block (warps without rows skip it)
    const bool has_rows = (int)(tid & ~31) < nk;
    for (int j = 0; has_rows && j < nhh; ++j) {
        const T *xb = x + sHH[j].base;
        const A g = sHH[j].g;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = tid + i * kThreads;
            if constexpr (TR) {
                if (act[i]) acc[i] += g * A(x_kept(x, map, sHH[j].base + r));
            } else {
                if (r < nk) acc[i] += g * A(__ldg(xb + r));
            }
        }
    }

    // high <-> low: stage each neighbouring block once (plain loads between two
    // barriers; measured faster on GB300 than a cp.async ring fetching ahead)
    for (int t = 0; t < H; ++t) {
        const uint64_t b2 = sMX[t];
        if (b2 == ~0ull) continue;            // CTA-uniform
        const bool occ_t = (h >> t) & 1ull;
        const int n2 = (int)__ldg(binom + L * kBinomStride + (occ_t ? k + 1 : k - 1));
        __syncthreads();
        for (int r = tid; r < n2; r += kThreads) sxn[r] = TR ? x_kept(x, map, b2 + r) : x[b2 + r];
        __syncthreads();
        const int go = L + t;
        if (occ_t) {                           // pair: high orbit go -> empty low orbit q
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (act[i]) {
                    const uint32_t l = lr[i];
                    A a = acc[i];
                    uint32_t emp = ~l & maskL;
                    for (int v = 0; v < L - k; ++v) {
                        const int q = __ffs(emp) - 1;
                        emp &= emp - 1;
                        a += sG[q * omega + go] * A(sxn[sRank[l | (1u << q)]]);
                    }
                    acc[i] = a;
                }
            }
        } else {                               // pair: occupied low orbit o -> high orbit go
#pragma unroll
            for (int i = 0; i < R; ++i) {
                if (act[i]) {
                    const uint32_t l = lr[i];
                    A a = acc[i];
                    uint32_t occ = l;
                    for (int u = 0; u < k; ++u) {
                        const int o = __ffs(occ) - 1;
                        occ &= occ - 1;
                        a += sG[go * omega + o] * A(sxn[sRank[l ^ (1u << o)]]);
                    }
                    acc[i] = a;
                }
            }
        }
    }

#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * kThreads;
        if constexpr (TR) {
            if (r < nk) {                     // dropped rows are not part of y
                const int32_t m = __ldg(map + base + r);
                if (m >= 0) y[m] = T(acc[i]);
            }
        } else {
            if (r < nk) y[base + r] = T(acc[i]);
        }
    }
    // (truncated: a dropped row has sx = 0, so it adds nothing to the dot)
    if (swdot) warp_dot<T, A, R>(acc, sx, nk, swdot);
}

template <typename T, typename A, int R, bool TR>
__global__ void __launch_bounds__(kThreads)
hx_kernel(const Blocks B, const A *__restrict__ Gg, const A *__restrict__ dg,
          const T *__restrict__ x, T *__restrict__ y, Tickets *tk, const int *__restrict__ skip,
          double *blk_part, double *dot_out)
{
    if (skip && *skip) return;                    // CTA-uniform
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_next[2];
    __shared__ double sred[kThreads / 32];
    __shared__ double swdot[kThreads / 32];
    const int omega = B.omega, L = B.L, H = B.H, N = B.n;
    // a truncated space walks only the blocks that hold kept states
    const int64_t nb = TR ? B.kept_nblocks : B.nblocks;
    const uint64_t *__restrict__ bh = TR ? B.kept_blk_h : B.blk_h;
    const uint64_t *__restrict__ bbase = TR ? B.kept_blk_base : B.blk_base;
    const Layout lay = layout<T, A>(omega, L, H, B.max_block, B.max_hh);
    A *sG = reinterpret_cast<A *>(smem + lay.G);
    A *sd = reinterpret_cast<A *>(smem + lay.d);
    uint16_t *sRank = reinterpret_cast<uint16_t *>(smem + lay.rank);
    T *sx = reinterpret_cast<T *>(smem + lay.x);
    T *sxn = reinterpret_cast<T *>(smem + lay.xn);
    HHop<A> *sHH = reinterpret_cast<HHop<A> *>(smem + lay.hh);
    uint64_t *sMX = reinterpret_cast<uint64_t *>(smem + lay.mx);
    const int tid = threadIdx.x;

    for (int i = tid; i < omega * omega; i += kThreads) sG[i] = Gg[i];
    for (int i = tid; i < omega; i += kThreads) sd[i] = dg[i];
    for (int i = tid; i < (1 << L); i += kThreads) sRank[i] = B.rankL[i];

    // the next block index is taken one block ahead (slot it ^ 1), so one
    // barrier per block both frees shared memory and publishes the index
    if (tid == 0) s_next[0] = (long long)atomicAdd(&tk->hx_next, 1ull);
    long long prev = -1;
    for (int it = 0;; it ^= 1) {
        __syncthreads();                          // smem of the previous block is free
        const long long b = s_next[it];
        if (tid == 0) {
            block_sum_deferred(blk_part, prev, swdot);
            if (b < nb) s_next[it ^ 1] = (long long)atomicAdd(&tk->hx_next, 1ull);
        }
        if (b >= nb) break;

        hx_block<T, A, R, TR>(omega, L, H, N, __ldg(bh + b), __ldg(bbase + b), B.lowword, B.binom,
                              sG, sd, sRank, sx, sxn, sHH, sMX, x, y, blk_part ? swdot : nullptr, B.kept_map);
        prev = b;
    }
    hx_finish(tk, nb, blk_part, dot_out, sred);
}

// ---- batched: blocks of many problems in one launch ----------------------------
// The global block list is sorted by problem.  A CTA reloads the problem's G, d
// and rank table only when the next block it takes belongs to another problem;
// problems flagged in skip[] (converged, or broken down in this cycle) are
// passed over.
template <typename T, typename A, int R>
__global__ void __launch_bounds__(kThreads)
hx_batch_kernel(const BatchBlocks BB, const A *__restrict__ Gall, const A *__restrict__ dall,
                const T *__restrict__ x, T *__restrict__ y, unsigned long long *counter,
                const int *__restrict__ skip, int skip_stride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_next;
    const Layout lay = layout<T, A>(BB.max_omega, BB.max_L, BB.max_H, BB.max_block, BB.max_hh);
    A *sG = reinterpret_cast<A *>(smem + lay.G);
    A *sd = reinterpret_cast<A *>(smem + lay.d);
    uint16_t *sRank = reinterpret_cast<uint16_t *>(smem + lay.rank);
    T *sx = reinterpret_cast<T *>(smem + lay.x);
    T *sxn = reinterpret_cast<T *>(smem + lay.xn);
    HHop<A> *sHH = reinterpret_cast<HHop<A> *>(smem + lay.hh);
    uint64_t *sMX = reinterpret_cast<uint64_t *>(smem + lay.mx);
    const int tid = threadIdx.x;
    int cur = -1;
    BatchDesc dsc{};

    for (;;) {
        __syncthreads();                          // smem of the previous block is free
        if (tid == 0) s_next = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long b = s_next;
        if (b >= BB.nblocks) break;
        const int pb = (int)__ldg(BB.blk_prob + b);
        if (skip && skip[(int64_t)pb * skip_stride]) continue;   // CTA-uniform
        if (pb != cur) {
            dsc = BB.desc[pb];
            const A *G = Gall + dsc.g_off;
            const A *d = dall + dsc.d_off;
            for (int i = tid; i < dsc.omega * dsc.omega; i += kThreads) sG[i] = G[i];
            for (int i = tid; i < dsc.omega; i += kThreads) sd[i] = d[i];
            const uint16_t *rk = BB.rankL_all + dsc.tab_off;
            for (int i = tid; i < (1 << dsc.L); i += kThreads) sRank[i] = rk[i];
            cur = pb;
            __syncthreads();
        }
        hx_block<T, A, R>(dsc.omega, dsc.L, dsc.omega - dsc.L, dsc.n, __ldg(BB.blk_h + b), __ldg(BB.blk_base + b),
                          BB.lowword_all + dsc.tab_off, BB.binom, sG, sd, sRank, sx, sxn, sHH, sMX,
                          x + dsc.vec_off, y + dsc.vec_off, nullptr);
    }
    // the last CTA to finish returns the block counter to zero (arrive_last
    // resets its own ticket), so the next launch needs no memset
    if (arrive_last(counter + 1) && tid == 0) counter[0] = 0ull;
}

// ---- variant 2: every neighbouring block of the high<->low hops staged at once --
struct Layout2 {
    size_t g, gs, ge, d, rank, low, bin, x, xn, hh, occ, emp, total;
};

template <typename T, typename A>
__host__ __device__ inline Layout2 layout2(int omega, int L, int H, int N, int max_block, int max_hh,
                                          int max_stage)
{
    Layout2 s;
    size_t off = 0;
    const int h1 = H > 0 ? H : 1;
    s.g = off;    off = align16(off + sizeof(A) * omega * omega);
    s.gs = off;   off = align16(off + sizeof(A) * h1 * L);
    s.ge = off;   off = align16(off + sizeof(A) * h1 * L);
    s.d = off;    off = align16(off + sizeof(A) * omega);
    s.rank = off; off = align16(off + sizeof(uint16_t) * (size_t(1) << L));
    s.low = off;  off = align16(off + sizeof(uint16_t) * (size_t(1) << L));
    s.bin = off;  off = align16(off + sizeof(uint64_t) * h1 * (N + 1));
    s.x = off;    off = align16(off + sizeof(T) * max_block);
    s.xn = off;   off = align16(off + sizeof(T) * (size_t)(max_stage > 0 ? max_stage : 1));
    s.hh = off;   off = align16(off + sizeof(HHop<A>) * (max_hh > 0 ? max_hh : 1));
    s.occ = off;  off = align16(off + sizeof(uint64_t) * h1);
    s.emp = off;  off = align16(off + sizeof(uint64_t) * h1);
    s.total = off;
    return s;
}

// block_base with the binomials of the high orbits in shared memory:
// sBin[p * (N + 1) + m] = C(L + p, m)
__device__ __forceinline__ uint64_t block_base_s(uint64_t h, int N, const uint64_t *sBin)
{
    int ord = N - __popcll(h);
    uint64_t s = 0;
    while (h) {
        const int p = __ffsll((long long)h) - 1;
        h &= h - 1;
        ++ord;
        s += sBin[p * (N + 1) + ord];
    }
    return s;
}

// asynchronous copy of one 4- or 8-byte element global -> shared (no register
// round trip, so a thread issues all its copies before any has landed)
template <typename T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src)
{
    static_assert(sizeof(T) == 4 || sizeof(T) == 8, "cp.async element of 4 or 8 bytes");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Shared-memory view of variant 2 (one CTA's dynamic shared memory)
template <typename T, typename A>
struct Smem2 {
    A *G, *GS, *GE, *d;
    uint16_t *rank, *low;
    uint64_t *bin, *occ, *emp;
    T *x, *xn;
    HHop<A> *hh;
    __device__ Smem2(unsigned char *smem, const Layout2 &lay)
        : G(reinterpret_cast<A *>(smem + lay.g)), GS(reinterpret_cast<A *>(smem + lay.gs)),
          GE(reinterpret_cast<A *>(smem + lay.ge)), d(reinterpret_cast<A *>(smem + lay.d)),
          rank(reinterpret_cast<uint16_t *>(smem + lay.rank)), low(reinterpret_cast<uint16_t *>(smem + lay.low)),
          bin(reinterpret_cast<uint64_t *>(smem + lay.bin)), occ(reinterpret_cast<uint64_t *>(smem + lay.occ)),
          emp(reinterpret_cast<uint64_t *>(smem + lay.emp)), x(reinterpret_cast<T *>(smem + lay.x)),
          xn(reinterpret_cast<T *>(smem + lay.xn)), hh(reinterpret_cast<HHop<A> *>(smem + lay.hh))
    {
    }
};

// One problem's tables into shared memory, read for the whole launch (or, in
// the batch, until the problem changes): G, d = 2e + diag(G), the rank and
// low-word tables of L-bit words, and the binomials C(L + p, m) of the high
// orbits (p < H, m <= N) that block_base_s adds up.
template <typename T, typename A>
__device__ __forceinline__ void load_tables2(const Smem2<T, A> &s, int omega, int L, int H, int N,
                                             const A *__restrict__ G, const A *__restrict__ d,
                                             const uint16_t *__restrict__ rankL, const uint16_t *__restrict__ lowword,
                                             const uint64_t *__restrict__ binom)
{
    const int tid = threadIdx.x;
    for (int i = tid; i < omega * omega; i += kThreads) s.G[i] = G[i];
    for (int i = tid; i < omega; i += kThreads) s.d[i] = d[i];
    for (int i = tid; i < (1 << L); i += kThreads) {
        s.rank[i] = rankL[i];
        s.low[i] = lowword[i];
    }
    for (int i = tid; i < (H > 0 ? H : 1) * (N + 1); i += kThreads) {
        const int p = i / (N + 1), m = i - p * (N + 1);
        s.bin[i] = __ldg(binom + (L + p) * kBinomStride + m);
    }
}

// One basis block (high word h, first index base) of y = H x in variant 2.
// x and y point at the problem's own vector; s holds its tables.  Called by
// every thread of the CTA after a barrier that frees the previous block's
// shared memory; it contains two barriers.  Any cp.async the caller issued
// before is completed by the first of them.  swdot (nullable): x^T y per warp.
template <typename T, typename A, int R>
__device__ __forceinline__ void hx2_block(const Smem2<T, A> &s, const int omega, const int L, const int H,
                                          const int N, const uint64_t h, const uint64_t base,
                                          const T *__restrict__ x, T *__restrict__ y, double *swdot)
{
    const int tid = threadIdx.x;
    const uint32_t maskL = (1u << L) - 1u;
    const uint64_t maskH = (H >= 64) ? ~0ull : ((1ull << H) - 1ull);
    const int ph = __popcll(h);
    const int k = N - ph;
    const int nemp = H - ph;
    const int nhh = ph * nemp;
    // block sizes C(L, k), C(L, k+1), C(L, k-1) from row p = 0 of s.bin
    // (k + 1 <= N whenever a block h - o exists, i.e. ph > 0)
    const int nk = (int)s.bin[k];
    const int n_up = (k < L && ph > 0) ? (int)s.bin[k + 1] : 0;
    const int n_dn = (k > 0 && nemp > 0) ? (int)s.bin[k - 1] : 0;
    int lo_off = 0;                               // words of popcount k start here in s.low
    for (int j = 0; j < k; ++j) lo_off += (int)s.bin[j];
    const uint16_t *lw = s.low + lo_off;
    T *sxn = s.xn;
    T *sxd = sxn + ph * n_up;                     // staged blocks h + e start here

    for (int r = tid; r < nk; r += kThreads) cp_async_elem(s.x + r, x + base + r);
    cp_async_commit();

    for (int t = tid; t < nhh; t += kThreads) {
        const int a = t / nemp, c = t - a * nemp;
        const int o = nth_set_bit(h, a);
        const int q = nth_set_bit(~h & maskH, c);
        s.hh[t].base = block_base_s(h ^ (1ull << o) ^ (1ull << q), N, s.bin);
        s.hh[t].g = s.G[(L + q) * omega + (L + o)];
    }
    for (int t = tid; t < H; t += kThreads) {
        const uint64_t bit = 1ull << t;
        if (h & bit) {
            const int j = __popcll(h & (bit - 1));
            s.occ[j] = n_up ? block_base_s(h ^ bit, N, s.bin) : 0;
            for (int e = 0; e < L; ++e) s.GS[j * L + e] = s.G[e * omega + L + t];
        } else {
            const int j = __popcll(~h & maskH & (bit - 1));
            s.emp[j] = n_dn ? block_base_s(h | bit, N, s.bin) : 0;
            for (int o = 0; o < L; ++o) s.GE[j * L + o] = s.G[(L + t) * omega + o];
        }
    }
    cp_async_wait_all();
    __syncthreads();                              // own block, hop tables and slot bases visible

    if (n_up)
        for (int j = 0; j < ph; ++j) {
            const T *src = x + s.occ[j];
            T *dst = sxn + j * n_up;
            for (int r = tid; r < n_up; r += kThreads) cp_async_elem(dst + r, src + r);
        }
    if (n_dn)
        for (int j = 0; j < nemp; ++j) {
            const T *src = x + s.emp[j];
            T *dst = sxd + j * n_dn;
            for (int r = tid; r < n_dn; r += kThreads) cp_async_elem(dst + r, src + r);
        }
    cp_async_commit();

    A Dh = A(0);
    for (uint64_t w = h; w; w &= w - 1) Dh += s.d[L + __ffsll((long long)w) - 1];

    uint32_t lr[R];
    A acc[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * kThreads;
        lr[i] = 0;
        acc[i] = A(0);
        if (r < nk) {
            const uint32_t l = lw[r];
            lr[i] = l;
            A D = A(0);
            for (uint32_t w = l; w; w &= w - 1) D += s.d[__ffs(w) - 1];
            acc[i] = (D + Dh) * A(s.x[r]);
        }
    }

    // low -> low
    if (k > 0 && k < L) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (tid + i * kThreads < nk) {
                const uint32_t l = lr[i];
                A a = acc[i];
                uint32_t occ = l;
                for (int u = 0; u < k; ++u) {
                    const int o = __ffs(occ) - 1;
                    occ &= occ - 1;
                    const uint32_t lo = l ^ (1u << o);
                    const A *gcol = s.G + o;
                    uint32_t emp = ~l & maskL;
                    for (int v = 0; v < L - k; ++v) {
                        const int q = __ffs(emp) - 1;
                        emp &= emp - 1;
                        a += gcol[q * omega] * A(s.x[s.rank[lo | (1u << q)]]);
                    }
                }
                acc[i] = a;
            }
        }
    }

    // high -> high: same offsets in the target block (warps without rows skip it)
    const bool has_rows = (int)(tid & ~31) < nk;
    for (int j = 0; has_rows && j < nhh; ++j) {
        const T *xb = x + s.hh[j].base;
        const A g = s.hh[j].g;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = tid + i * kThreads;
            if (r < nk) acc[i] += g * A(__ldg(xb + r));
        }
    }
    cp_async_wait_all();
    __syncthreads();                              // staged neighbour blocks visible

    // high -> low: pair from occupied high orbit L+t to empty low orbit e;
    // the target offset rank(l + e) is the same in every staged block
    if (n_up) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = tid + i * kThreads;
            if (r < nk) {
                const uint32_t l = lr[i];
                A a = acc[i];
                for (uint32_t w = ~l & maskL; w; w &= w - 1) {
                    const int e = __ffs(w) - 1;
                    const A *g = s.GS + e;
                    const T *xp = sxn + s.rank[l | (1u << e)];
                    for (int j = 0; j < ph; ++j) a += g[j * L] * A(xp[j * n_up]);
                }
                acc[i] = a;
            }
        }
    }
    // low -> high: pair from occupied low orbit o to empty high orbit L+t
    if (n_dn) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int r = tid + i * kThreads;
            if (r < nk) {
                const uint32_t l = lr[i];
                A a = acc[i];
                for (uint32_t w = l; w; w &= w - 1) {
                    const int o = __ffs(w) - 1;
                    const A *g = s.GE + o;
                    const T *xp = sxd + s.rank[l ^ (1u << o)];
                    for (int j = 0; j < nemp; ++j) a += g[j * L] * A(xp[j * n_dn]);
                }
                acc[i] = a;
            }
        }
    }

#pragma unroll
    for (int i = 0; i < R; ++i) {
        const int r = tid + i * kThreads;
        if (r < nk) y[base + r] = T(acc[i]);
    }
    if (swdot) warp_dot<T, A, R>(acc, s.x, nk, swdot);
}

// Same product as hx_kernel.  Differences: all ph blocks h - o (k+1 low pairs)
// and all H-ph blocks h + e (k-1) are staged together; the coefficients of the
// high<->low hops are laid out per staged block (G_{e, L+t} for block h - t at
// row t of sGS, G_{L+t, o} for block h + t in sGE), so for each row and low
// orbit the innermost loop runs over the staged blocks with one coefficient
// load, one gather and one FMA.
//
// Latency: G, d, the rank and low-word tables and the binomials of the high
// orbits live in shared memory for the whole launch, so the per-block tables
// need no global loads; the block's own x and its neighbours arrive through
// cp.async, issued before the table setup and before the low->low and
// high->high hops respectively, so their latency overlaps that work; thread 0
// takes the next block index and copies its (h, base) into shared memory one
// block ahead.  FP32: at most 40 registers, so that six CTAs fit an SM when
// shared memory allows.
template <typename T, typename A, int R>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 6 : 4)
hx2_kernel(const Blocks B, const A *__restrict__ Gg, const A *__restrict__ dg,
           const T *__restrict__ x, T *__restrict__ y, Tickets *tk, const int *__restrict__ skip,
           double *blk_part, double *dot_out)
{
    if (skip && *skip) return;                    // CTA-uniform
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_idx[2];
    __shared__ __align__(8) uint64_t s_h[2], s_base[2];
    __shared__ double sred[kThreads / 32];
    __shared__ double swdot[kThreads / 32];
    const int omega = B.omega, L = B.L, H = B.H, N = B.n;
    const Smem2<T, A> s(smem, layout2<T, A>(omega, L, H, N, B.max_block, B.max_hh, B.max_stage));
    const int tid = threadIdx.x;
    load_tables2<T, A>(s, omega, L, H, N, Gg, dg, B.rankL, B.lowword, B.binom);

    // block schedule: slot it holds (index, h, base) of the block of iteration
    // it.  Thread 0 holds the index of the next block in nb1; during the
    // current block it copies that block's (h, base) into slot it ^ 1 with
    // cp.async (completed by the first barrier of hx2_block) and takes the
    // index after it from the counter, so neither latency delays a block.
    // (Block counts are below 2^31: build_tables rejects more blocks.)
    const int nblocks = (int)B.nblocks;
    int nb1 = 0;
    if (tid == 0) {
        const int b0 = (int)atomicAdd(&tk->hx_next, 1ull);
        s_idx[0] = b0;
        if (b0 < nblocks) {
            s_h[0] = __ldg(B.blk_h + b0);
            s_base[0] = __ldg(B.blk_base + b0);
            nb1 = (int)atomicAdd(&tk->hx_next, 1ull);
        }
    }
    long long prev = -1;
    for (int it = 0;; it ^= 1) {
        __syncthreads();                          // smem of the previous block is free; slot it visible
        const int b = s_idx[it];
        int nb2 = 0;
        if (tid == 0) {
            block_sum_deferred(blk_part, prev, swdot);
            if (b < nblocks && nb1 < nblocks) {
                cp_async_elem(&s_h[it ^ 1], B.blk_h + nb1);
                cp_async_elem(&s_base[it ^ 1], B.blk_base + nb1);
                nb2 = (int)atomicAdd(&tk->hx_next, 1ull);
            }
        }
        if (b >= nblocks) break;
        hx2_block<T, A, R>(s, omega, L, H, N, s_h[it], s_base[it], x, y, blk_part ? swdot : nullptr);
        prev = b;
        if (tid == 0) {                           // publish the next block (read after the barrier)
            s_idx[it ^ 1] = nb1;
            nb1 = nb2;
        }
    }
    hx_finish(tk, B.nblocks, blk_part, dot_out, sred);
}

// ---- variant 3: no staging rounds; hop tables in O(1) per entry ------------------
// Variants 1 and 2 stage neighbour blocks in shared memory, which pays when
// blocks are large (half filling).  Far from half filling most blocks hold a
// few rows (C(12,0..1) = 1..12 at Omega=38, N=10), and there variant 1's H
// staging rounds (each a memory latency plus two barriers) and the per-entry
// block_base loops of the hop tables dominate.  Variant 3 gathers every
// target straight from global memory (L2) with one barrier per block, and
// builds the hop tables from prefix sums of binomials over the block's high
// pairs.  With P_1 < ... < P_ph the occupied high orbits (ordinals k+1..N),
//   A_i = C(L+P_i, k+i), B_i = C(L+P_i, k+i-1), C_i = C(L+P_i, k+i+1)
// and SA, SB, SC their prefix sums (SA[ph] = base(h)):
//   base(h - P_a + q) = SA[ph] - (SA[b] - SA[a-1]) + (SB[b] - SB[a]) + C(L+q, k+b)   (a <= b)
//                     = SA[ph] - (SA[a] - SA[b]) + (SC[a-1] - SC[b]) + C(L+q, k+b+1)  (a > b)
//   base(h - P_a)     = SC[a-1] + SA[ph] - SA[a]              (k+1 low pairs)
//   base(h + q)       = SB[b] + C(L+q, k+b) + SA[ph] - SA[b]   (k-1 low pairs)
// with q an empty high orbit and b the number of occupied high orbits below q:
// the pairs between the moved ones change ordinal by one, the others keep it.
struct Layout3 {
    size_t g, d, rank, bin, x, hp, hg, xo, xe, gs, ge, sa, sb, sc, pos, emp, eb, part, total;
};

template <typename T, typename A>
__host__ __device__ inline Layout3 layout3(int omega, int L, int H, int N, int max_block, int max_hh)
{
    Layout3 s;
    size_t off = 0;
    const int h1 = H > 0 ? H : 1;
    const int hh1 = max_hh > 0 ? max_hh : 1;
    s.g = off;    off = align16(off + sizeof(A) * omega * omega);
    s.d = off;    off = align16(off + sizeof(A) * omega);
    s.rank = off; off = align16(off + sizeof(uint16_t) * (size_t(1) << L));
    s.bin = off;  off = align16(off + sizeof(uint64_t) * h1 * (N + 2));
    s.x = off;    off = align16(off + sizeof(T) * max_block);
    s.hp = off;   off = align16(off + sizeof(const T *) * hh1);
    s.hg = off;   off = align16(off + sizeof(A) * hh1);
    s.xo = off;   off = align16(off + sizeof(const T *) * h1);
    s.xe = off;   off = align16(off + sizeof(const T *) * h1);
    s.gs = off;   off = align16(off + sizeof(A) * h1 * L);
    s.ge = off;   off = align16(off + sizeof(A) * h1 * L);
    s.sa = off;   off = align16(off + sizeof(uint64_t) * (h1 + 1));
    s.sb = off;   off = align16(off + sizeof(uint64_t) * (h1 + 1));
    s.sc = off;   off = align16(off + sizeof(uint64_t) * (h1 + 1));
    s.pos = off;  off = align16(off + sizeof(int) * h1);
    s.emp = off;  off = align16(off + sizeof(int) * h1);
    s.eb = off;   off = align16(off + sizeof(int) * h1);
    s.part = off; off = align16(off + sizeof(A) * kThreads);
    s.total = off;
    return s;
}

// Shared-memory view of variant 3.  Per block: hp/hg the high->high targets
// (pointer to the target block, coefficient); xo[a] the block h - P_a and
// xe[c] the block h + q_c (pointers); gs[a*L + e] = G_{e, L+P_a} and
// ge[c*L + o] = G_{L+q_c, o}, the coefficients of the high<->low hops.
template <typename T, typename A>
struct Smem3 {
    A *G, *d, *hg, *gs, *ge, *part;
    uint16_t *rank;
    uint64_t *bin, *sa, *sb, *sc;
    int *pos, *emp, *eb;
    T *x;
    const T **hp, **xo, **xe;
    __device__ Smem3(unsigned char *m, const Layout3 &l)
        : G(reinterpret_cast<A *>(m + l.g)), d(reinterpret_cast<A *>(m + l.d)), hg(reinterpret_cast<A *>(m + l.hg)),
          gs(reinterpret_cast<A *>(m + l.gs)), ge(reinterpret_cast<A *>(m + l.ge)),
          part(reinterpret_cast<A *>(m + l.part)), rank(reinterpret_cast<uint16_t *>(m + l.rank)),
          bin(reinterpret_cast<uint64_t *>(m + l.bin)), sa(reinterpret_cast<uint64_t *>(m + l.sa)),
          sb(reinterpret_cast<uint64_t *>(m + l.sb)), sc(reinterpret_cast<uint64_t *>(m + l.sc)),
          pos(reinterpret_cast<int *>(m + l.pos)), emp(reinterpret_cast<int *>(m + l.emp)),
          eb(reinterpret_cast<int *>(m + l.eb)), x(reinterpret_cast<T *>(m + l.x)),
          hp(reinterpret_cast<const T **>(m + l.hp)), xo(reinterpret_cast<const T **>(m + l.xo)),
          xe(reinterpret_cast<const T **>(m + l.xe))
    {
    }
};

// Small blocks (at most 32 rows, far from half filling): lane r of every warp
// takes row r, and warp w the hops of class index w, w + 8, ...; warp 0 adds
// the eight partial sums in warp order (a fixed order).  acc[0] of warp 0
// holds the row's diagonal and low->low terms on entry and the row's y on
// exit; y (of type TY) is written here.
template <typename T, typename A, int R, typename TY>
__device__ __forceinline__ void hx3_small(const Smem3<T, A> &s, const int L, const int k, const int ph,
                                          const int nemp, const int nhh, const uint64_t base,
                                          const uint16_t *__restrict__ lw, TY *__restrict__ y, const int nk,
                                          A (&acc)[R])
{
    constexpr int kW = kThreads / 32;
    const int tid = threadIdx.x, w = tid >> 5, r = tid & 31;
    const uint32_t maskL = (1u << L) - 1u;
    A a = (w == 0) ? acc[0] : A(0);
    if (r < nk) {
        const uint32_t l = __ldg(lw + r);
#pragma unroll 2
        for (int j = w; j < nhh; j += kW) a += s.hg[j] * A(__ldg(s.hp[j] + r));
        if (k < L)
            for (int ai = w; ai < ph; ai += kW) {
                const T *xb = s.xo[ai];
                const A *g = s.gs + ai * L;
                uint32_t em = ~l & maskL;
                for (int t = 0; t < L - k; ++t) {
                    const int e = __ffs(em) - 1;
                    em &= em - 1;
                    a += g[e] * A(__ldg(xb + s.rank[l | (1u << e)]));
                }
            }
        if (k > 0)
            for (int c = w; c < nemp; c += kW) {
                const T *xb = s.xe[c];
                const A *g = s.ge + c * L;
                uint32_t oc = l;
                for (int t = 0; t < k; ++t) {
                    const int o = __ffs(oc) - 1;
                    oc &= oc - 1;
                    a += g[o] * A(__ldg(xb + s.rank[l ^ (1u << o)]));
                }
            }
    }
    s.part[tid] = a;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i) acc[i] = A(0);
    if (w == 0 && r < nk) {
        A t = A(0);
#pragma unroll
        for (int q = 0; q < kW; ++q) t += s.part[q * 32 + r];
        acc[0] = t;
        y[base + r] = TY(t);
    }
}

// The rows of one block in variant 3 (RR rows per thread): diagonal, low->low
// from the staged block, then the gathers; writes y and the fused dot.
template <typename T, typename A, int RR, bool DEEP, typename TY>
__device__ __forceinline__ void hx3_rows(const Smem3<T, A> &s, const int omega, const int L, const uint64_t h,
                                         const uint64_t base, const uint16_t *__restrict__ lw,
                                         TY *__restrict__ y, double *swdot, const int k, const int ph,
                                         const int nemp, const int nhh, const int nk)
{
    const int tid = threadIdx.x;
    const uint32_t maskL = (1u << L) - 1u;
    A Dh = A(0);
    for (uint64_t w = h; w; w &= w - 1) Dh += s.d[L + __ffsll((long long)w) - 1];
    uint32_t lr[RR];
    A acc[RR];
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        const int r = tid + i * kThreads;
        lr[i] = 0;
        acc[i] = A(0);
        if (r < nk) {
            const uint32_t l = __ldg(lw + r);
            lr[i] = l;
            A D = A(0);
            for (uint32_t w = l; w; w &= w - 1) D += s.d[__ffs(w) - 1];
            acc[i] = (D + Dh) * A(s.x[r]);
            // low -> low (own block, shared memory)
            A a = acc[i];
            uint32_t oc = l;
            for (int u = 0; u < k; ++u) {
                const int o = __ffs(oc) - 1;
                oc &= oc - 1;
                const uint32_t lo = l ^ (1u << o);
                const A *gcol = s.G + o;
                uint32_t em = ~l & maskL;
                for (int v = 0; v < L - k; ++v) {
                    const int q = __ffs(em) - 1;
                    em &= em - 1;
                    a += gcol[q * omega] * A(s.x[s.rank[lo | (1u << q)]]);
                }
            }
            acc[i] = a;
        }
    }
    if (nk <= 32) {                               // block-uniform
        hx3_small<T, A, RR>(s, L, k, ph, nemp, nhh, base, lw, y, nk, acc);
        if (swdot) warp_dot<T, A, RR>(acc, s.x, nk, swdot);
        return;
    }
    // warps without a row of this block skip the gathers (warp-uniform)
    if ((int)(tid & ~31) < nk) {
        // high -> high: same offsets in the target block (coalesced).  Deep
        // form: the gathers of a group of kHH hops are issued before their
        // multiply-adds, so each warp has that many requests in flight per
        // memory latency (pays far from half filling, where x is in DRAM and
        // a thread has one row); lean form: a plain unrolled loop (fewer
        // instructions, which pays where the kernel is issue-bound).
        constexpr int kHH = 16 / RR;
        bool rv[RR];
#pragma unroll
        for (int i = 0; i < RR; ++i) rv[i] = tid + i * kThreads < nk;
        if constexpr (!DEEP) {
#pragma unroll 4
            for (int j = 0; j < nhh; ++j) {
                const T *xb = s.hp[j];
                const A g = s.hg[j];
#pragma unroll
                for (int i = 0; i < RR; ++i)
                    if (rv[i]) acc[i] += g * A(__ldg(xb + tid + i * kThreads));
            }
        }
        for (int j0 = 0; DEEP && j0 < nhh; j0 += kHH) {
            T v[kHH][RR];
#pragma unroll
            for (int u = 0; u < kHH; ++u) {
                const bool ok = j0 + u < nhh;
                const T *xb = s.hp[ok ? j0 + u : 0];
#pragma unroll
                for (int i = 0; i < RR; ++i) v[u][i] = (ok && rv[i]) ? __ldg(xb + tid + i * kThreads) : T(0);
            }
#pragma unroll
            for (int u = 0; u < kHH; ++u) {
                const A g = (j0 + u < nhh) ? s.hg[j0 + u] : A(0);
#pragma unroll
                for (int i = 0; i < RR; ++i) acc[i] += g * A(v[u][i]);
            }
        }
#pragma unroll
        for (int i = 0; i < RR; ++i) {
            if (tid + i * kThreads >= nk) continue;
            const uint32_t l = lr[i];
            A a = acc[i];
            // high -> low: occupied high orbit P_a to empty low orbit e (block h - P_a)
            if (k < L) {
                uint32_t em = ~l & maskL;
                for (int t = 0; t < L - k; ++t) {
                    const int e = __ffs(em) - 1;
                    em &= em - 1;
                    const uint32_t off = s.rank[l | (1u << e)];
                    const A *g = s.gs + e;
                    if constexpr (!DEEP) {
#pragma unroll 4
                        for (int ai = 0; ai < ph; ++ai) a += g[ai * L] * A(__ldg(s.xo[ai] + off));
                        continue;
                    }
                    for (int a0 = 0; a0 < ph; a0 += 8) {
                        T v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            v[u] = (a0 + u < ph) ? __ldg(s.xo[a0 + u] + off) : T(0);
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (a0 + u < ph) a += g[(a0 + u) * L] * A(v[u]);
                    }
                }
            }
            // low -> high: occupied low orbit o to empty high orbit q_c (block h + q_c)
            if (k > 0) {
                uint32_t oc = l;
                for (int t = 0; t < k; ++t) {
                    const int o = __ffs(oc) - 1;
                    oc &= oc - 1;
                    const uint32_t off = s.rank[l ^ (1u << o)];
                    const A *g = s.ge + o;
                    if constexpr (!DEEP) {
#pragma unroll 4
                        for (int c = 0; c < nemp; ++c) a += g[c * L] * A(__ldg(s.xe[c] + off));
                        continue;
                    }
                    for (int c0 = 0; c0 < nemp; c0 += 8) {
                        T v[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            v[u] = (c0 + u < nemp) ? __ldg(s.xe[c0 + u] + off) : T(0);
#pragma unroll
                        for (int u = 0; u < 8; ++u)
                            if (c0 + u < nemp) a += g[(c0 + u) * L] * A(v[u]);
                    }
                }
            }
            acc[i] = a;
        }
    }
#pragma unroll
    for (int i = 0; i < RR; ++i) {
        const int r = tid + i * kThreads;
        if (r < nk) y[base + r] = TY(acc[i]);
    }
    if (swdot) warp_dot<T, A, RR>(acc, s.x, nk, swdot);
}

// One basis block of y = H x in variant 3.  Called by every thread after a
// barrier that frees the previous block's shared memory.
template <typename T, typename A, int R, bool DEEP, typename TY>
__device__ __forceinline__ void hx3_block(const Smem3<T, A> &s, const int omega, const int L, const int H,
                                          const int N, const uint64_t h, const uint64_t base,
                                          const uint16_t *__restrict__ lowword, const T *__restrict__ x,
                                          TY *__restrict__ y, double *swdot)
{
    const int tid = threadIdx.x;
    const int ph = __popcll(h);
    const int k = N - ph;
    const int nemp = H - ph;
    const int nhh = ph * nemp;
    const int NB = N + 2;                         // row stride of s.bin: C(L + p, m), m <= N + 1
    const int nk = (int)s.bin[k];
    int lo_off = 0;
    for (int j = 0; j < k; ++j) lo_off += (int)s.bin[j];
    const uint16_t *lw = lowword + lo_off;

    for (int r = tid; r < nk; r += kThreads) s.x[r] = x[base + r];
    if (tid < 32) {                               // warp 0: positions and prefix sums of the high pairs
        const int lane = tid;
        const unsigned lt = (1u << lane) - 1u;
        uint64_t ca = 0, cb = 0, cc = 0;
        int cocc = 0, cemp = 0;
        for (int j0 = 0; j0 < H; j0 += 32) {
            const int j = j0 + lane;
            const bool in = j < H;
            const bool occ = in && ((h >> j) & 1ull);
            const unsigned bo = __ballot_sync(0xffffffffu, occ);
            const unsigned be = __ballot_sync(0xffffffffu, in && !occ);
            const int io = cocc + __popc(bo & lt);        // occupied high orbits below j
            uint64_t a = 0, b = 0, c = 0;
            if (occ) {
                const uint64_t *row = s.bin + j * NB;
                a = row[k + io + 1];
                b = row[k + io];
                c = row[k + io + 2];
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t ta = __shfl_up_sync(0xffffffffu, a, o);
                const uint64_t tb = __shfl_up_sync(0xffffffffu, b, o);
                const uint64_t tc = __shfl_up_sync(0xffffffffu, c, o);
                if (lane >= o) { a += ta; b += tb; c += tc; }
            }
            a += ca; b += cb; c += cc;
            if (occ) {
                s.sa[io + 1] = a;
                s.sb[io + 1] = b;
                s.sc[io + 1] = c;
                s.pos[io] = j;
            }
            if (in && !occ) {
                const int ie = cemp + __popc(be & lt);
                s.emp[ie] = j;
                s.eb[ie] = io;
            }
            ca = __shfl_sync(0xffffffffu, a, 31);
            cb = __shfl_sync(0xffffffffu, b, 31);
            cc = __shfl_sync(0xffffffffu, c, 31);
            cocc += __popc(bo);
            cemp += __popc(be);
        }
        if (lane == 0) s.sa[0] = s.sb[0] = s.sc[0] = 0ull;
    }
    __syncthreads();                              // prefix sums, positions, own block visible

    const uint64_t SA = s.sa[ph];                 // base(h)
    for (int t = tid; t < nhh; t += kThreads) {
        const int a1 = t / nemp + 1, c = t - (a1 - 1) * nemp;
        const int q = s.emp[c], b = s.eb[c];
        const uint64_t *row = s.bin + q * NB;
        const uint64_t bb = (a1 <= b) ? SA - (s.sa[b] - s.sa[a1 - 1]) + (s.sb[b] - s.sb[a1]) + row[k + b]
                                      : SA - (s.sa[a1] - s.sa[b]) + (s.sc[a1 - 1] - s.sc[b]) + row[k + b + 1];
        s.hp[t] = x + bb;
        s.hg[t] = s.G[(L + q) * omega + (L + s.pos[a1 - 1])];
    }
    for (int a = tid; a < ph; a += kThreads) s.xo[a] = x + ((k < L) ? s.sc[a] + SA - s.sa[a + 1] : 0ull);
    for (int c = tid; c < nemp; c += kThreads) {
        const int b = s.eb[c];
        s.xe[c] = x + ((k > 0) ? s.sb[b] + s.bin[s.emp[c] * NB + k + b] + SA - s.sa[b] : 0ull);
    }
    for (int i = tid; i < ph * L; i += kThreads) {
        const int a = i / L, e = i - a * L;
        s.gs[i] = s.G[e * omega + L + s.pos[a]];
    }
    for (int i = tid; i < nemp * L; i += kThreads) {
        const int c = i / L, o = i - c * L;
        s.ge[i] = s.G[(L + s.emp[c]) * omega + o];
    }
    __syncthreads();                              // hop tables visible
    // the row work, unrolled for the rows per thread this block needs
    const int rpt = (nk + kThreads - 1) / kThreads;
    if (rpt <= 1) hx3_rows<T, A, 1, DEEP>(s, omega, L, h, base, lw, y, swdot, k, ph, nemp, nhh, nk);
    else if (rpt <= 2)
        hx3_rows<T, A, (R < 2 ? R : 2), DEEP>(s, omega, L, h, base, lw, y, swdot, k, ph, nemp, nhh, nk);
    else if (rpt <= 4)
        hx3_rows<T, A, (R < 4 ? R : 4), DEEP>(s, omega, L, h, base, lw, y, swdot, k, ph, nemp, nhh, nk);
    else hx3_rows<T, A, R, DEEP>(s, omega, L, h, base, lw, y, swdot, k, ph, nemp, nhh, nk);
}

// OCC: resident CTAs per SM the register budget is cut for (4: 64 registers;
// 5: 48 registers, variant 5, more warps to hide the gathers' latency).
// TY: the type of y (double for float-float rows of an FP32 x)
template <typename T, typename A, int R, bool DEEP, int OCC = 4, typename TY = T>
__global__ void __launch_bounds__(kThreads, OCC)
hx3_kernel(const Blocks B, const A *__restrict__ Gg, const A *__restrict__ dg, const T *__restrict__ x,
           TY *__restrict__ y, Tickets *tk, const int *__restrict__ skip, double *blk_part, double *dot_out)
{
    if (skip && *skip) return;                    // CTA-uniform
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_next[2];
    __shared__ double sred[kThreads / 32];
    __shared__ double swdot[kThreads / 32];
    const int omega = B.omega, L = B.L, H = B.H, N = B.n;
    const Smem3<T, A> s(smem, layout3<T, A>(omega, L, H, N, B.max_block, B.max_hh));
    const int tid = threadIdx.x;
    for (int i = tid; i < omega * omega; i += kThreads) s.G[i] = Gg[i];
    for (int i = tid; i < omega; i += kThreads) s.d[i] = dg[i];
    for (int i = tid; i < (1 << L); i += kThreads) s.rank[i] = B.rankL[i];
    for (int i = tid; i < (H > 0 ? H : 1) * (N + 2); i += kThreads) {
        const int p = i / (N + 2), m = i - p * (N + 2);
        s.bin[i] = __ldg(B.binom + (L + p) * kBinomStride + m);
    }

    if (tid == 0) s_next[0] = (long long)atomicAdd(&tk->hx_next, 1ull);
    long long prev = -1;
    for (int it = 0;; it ^= 1) {
        __syncthreads();                          // smem of the previous block is free
        const long long b = s_next[it];
        if (tid == 0) {
            block_sum_deferred(blk_part, prev, swdot);
            if (b < B.nblocks) s_next[it ^ 1] = (long long)atomicAdd(&tk->hx_next, 1ull);
        }
        if (b >= B.nblocks) break;
        hx3_block<T, A, R, DEEP>(s, omega, L, H, N, __ldg(B.blk_h + b), __ldg(B.blk_base + b), B.lowword, x, y,
                           blk_part ? swdot : nullptr);
        prev = b;
    }
    hx_finish(tk, B.nblocks, blk_part, dot_out, sred);
}

// Batched form of variant 3: the blocks of many problems in one launch (the
// global block list is sorted by problem).  A CTA reloads the problem's G, d,
// rank table and binomials only when the next block it takes belongs to
// another problem; problems flagged in skip[] are passed over.  The last CTA
// returns both counters to zero.
template <typename T, typename A, int R, typename TY = T>
__global__ void __launch_bounds__(kThreads, 4)
hx3_batch_kernel(const BatchBlocks BB, const A *__restrict__ Gall, const A *__restrict__ dall,
                 const T *__restrict__ x, TY *__restrict__ y, unsigned long long *counter,
                 const int *__restrict__ skip, int skip_stride)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_next;
    const Smem3<T, A> s(smem, layout3<T, A>(BB.max_omega, BB.max_L, BB.max_H, BB.max_n, BB.max_block, BB.max_hh));
    const int tid = threadIdx.x;
    int cur = -1;
    BatchDesc dsc{};
    for (;;) {
        __syncthreads();                          // smem of the previous block is free
        if (tid == 0) s_next = (long long)atomicAdd(counter, 1ull);
        __syncthreads();
        const long long b = s_next;
        if (b >= BB.nblocks) break;
        const int pb = (int)__ldg(BB.blk_prob + b);
        if (skip && skip[(int64_t)pb * skip_stride]) continue;   // CTA-uniform
        if (pb != cur) {
            dsc = BB.desc[pb];
            const int om = dsc.omega, L = dsc.L, H = om - L, NB = dsc.n + 2;
            const A *G = Gall + dsc.g_off;
            const A *d = dall + dsc.d_off;
            for (int i = tid; i < om * om; i += kThreads) s.G[i] = G[i];
            for (int i = tid; i < om; i += kThreads) s.d[i] = d[i];
            const uint16_t *rk = BB.rankL_all + dsc.tab_off;
            for (int i = tid; i < (1 << L); i += kThreads) s.rank[i] = rk[i];
            for (int i = tid; i < (H > 0 ? H : 1) * NB; i += kThreads) {
                const int p = i / NB, m = i - p * NB;
                s.bin[i] = __ldg(BB.binom + (L + p) * kBinomStride + m);
            }
            cur = pb;
            __syncthreads();
        }
        hx3_block<T, A, R, false>(s, dsc.omega, dsc.L, dsc.omega - dsc.L, dsc.n, __ldg(BB.blk_h + b),
                                  __ldg(BB.blk_base + b), BB.lowword_all + dsc.tab_off, x + dsc.vec_off,
                                  y + dsc.vec_off, nullptr);
    }
    if (arrive_last(counter + 1) && tid == 0) counter[0] = 0ull;
}

constexpr size_t kSmemLimit = 200 * 1024;

// Variant 2 only on request (the autotuner's choice, or the caller's) and when
// its shared memory fits; which variant is faster depends on the problem and
// the block split (at Omega=24 variant 2 with L=11 in FP32, at Omega=32 variant 1).
template <typename T, typename A>
bool use_v2(const Blocks &B)
{
    if (B.variant != 2 || B.kept_map) return false;     // a truncated space runs variant 1
    return layout2<T, A>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh, B.max_stage).total <= kSmemLimit;
}

// Variant 3 (lean loops), 4 (deep gather groups) or 5 (lean loops, 5 CTAs per
// SM) on request, when the shared memory fits (full space only)
template <typename T, typename A>
bool use_v3(const Blocks &B)
{
    if ((B.variant < 3 || B.variant > 5) || B.kept_map) return false;
    return layout3<T, A>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh).total <= kSmemLimit;
}

template <typename T, typename A, int R>
const void *kernel_fn(const Blocks &B)
{
    if (B.kept_map) return (const void *)hx_kernel<T, A, R, true>;
    if (use_v3<T, A>(B))
        return B.variant == 4   ? (const void *)hx3_kernel<T, A, R, true>
               : B.variant == 5 ? (const void *)hx3_kernel<T, A, R, false, 5>
                                : (const void *)hx3_kernel<T, A, R, false>;
    return use_v2<T, A>(B) ? (const void *)hx2_kernel<T, A, R> : (const void *)hx_kernel<T, A, R, false>;
}

template <typename T, typename A>
size_t kernel_smem(const Blocks &B)
{
    if (use_v3<T, A>(B)) return layout3<T, A>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh).total;
    return use_v2<T, A>(B) ? layout2<T, A>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh, B.max_stage).total
                           : layout<T, A>(B.omega, B.L, B.H, B.max_block, B.max_hh).total;
}

template <typename T, typename A, int R>
cudaError_t launch_t(const Blocks &B, const A *G, const A *d, const void *x, void *y,
                     Tickets *tk, int grid, cudaStream_t st, const int *skip, const HxDot *dot)
{
    const size_t smem = kernel_smem<T, A>(B);
    const bool v2 = use_v2<T, A>(B);
    cudaError_t err = cudaFuncSetAttribute(kernel_fn<T, A, R>(B),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    double *bp = dot ? dot->blk_part : nullptr;
    double *out = dot ? dot->out : nullptr;
    if (B.kept_map)
        hx_kernel<T, A, R, true><<<grid, kThreads, smem, st>>>(B, G, d, static_cast<const T *>(x),
                                                               static_cast<T *>(y), tk, skip, bp, out);
    else if (use_v3<T, A>(B) && B.variant == 4)
        hx3_kernel<T, A, R, true><<<grid, kThreads, smem, st>>>(B, G, d, static_cast<const T *>(x),
                                                                static_cast<T *>(y), tk, skip, bp, out);
    else if (use_v3<T, A>(B) && B.variant == 5)
        hx3_kernel<T, A, R, false, 5><<<grid, kThreads, smem, st>>>(B, G, d, static_cast<const T *>(x),
                                                                    static_cast<T *>(y), tk, skip, bp, out);
    else if (use_v3<T, A>(B))
        hx3_kernel<T, A, R, false><<<grid, kThreads, smem, st>>>(B, G, d, static_cast<const T *>(x),
                                                                 static_cast<T *>(y), tk, skip, bp, out);
    else if (v2)
        hx2_kernel<T, A, R><<<grid, kThreads, smem, st>>>(B, G, d, static_cast<const T *>(x),
                                                          static_cast<T *>(y), tk, skip, bp, out);
    else
        hx_kernel<T, A, R, false><<<grid, kThreads, smem, st>>>(B, G, d, static_cast<const T *>(x),
                                                                static_cast<T *>(y), tk, skip, bp, out);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, typename A>
cudaError_t launch_prec(const Blocks &B, const A *G, const A *d, const void *x, void *y,
                        Tickets *tk, int grid, cudaStream_t st, const int *skip, const HxDot *dot)
{
    const int rows = (B.max_block + kThreads - 1) / kThreads;
    if (rows <= 1) return launch_t<T, A, 1>(B, G, d, x, y, tk, grid, st, skip, dot);
    if (rows <= 2) return launch_t<T, A, 2>(B, G, d, x, y, tk, grid, st, skip, dot);
    if (rows <= 4) return launch_t<T, A, 4>(B, G, d, x, y, tk, grid, st, skip, dot);
    return launch_t<T, A, 8>(B, G, d, x, y, tk, grid, st, skip, dot);
}

template <typename T, typename A>
int grid_prec(const Blocks &B)
{
    const size_t smem = kernel_smem<T, A>(B);
    const int rows = (B.max_block + kThreads - 1) / kThreads;
    const void *fn = rows <= 1 ? kernel_fn<T, A, 1>(B)
                   : rows <= 2 ? kernel_fn<T, A, 2>(B)
                   : rows <= 4 ? kernel_fn<T, A, 4>(B)
                               : kernel_fn<T, A, 8>(B);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)sms * per_sm;
    const int64_t nbk = B.kept_map ? B.kept_nblocks : B.nblocks;   // blocks a launch walks
    if (g > nbk) g = nbk;
    return (int)(g > 0 ? g : 1);
}

// ---- Monopole_Min / Monopole_Max / Posit_Min ---------------------------------
// Diagonal of each row summed over its occupied orbits in ascending orbit
// order (the oracle's order, so the values agree bit for bit).
__global__ void __launch_bounds__(kThreads)
monopole_kernel(const Blocks B, const double *__restrict__ d, double *__restrict__ part)
{
    double vmin = INFINITY, vmax = -INFINITY;
    long long imin = LLONG_MAX;
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b], base = B.blk_base[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        const uint16_t *lw = B.lowword + B.lo_off[k];
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            double D = 0.0;
            for (uint32_t w = lw[r]; w; w &= w - 1) D += d[__ffs(w) - 1];
            for (uint64_t w = h; w; w &= w - 1) D += d[B.L + __ffsll((long long)w) - 1];
            const long long idx = (long long)(base + r);
            if (D < vmin || (D == vmin && idx < imin)) { vmin = D; imin = idx; }
            if (D > vmax) vmax = D;
        }
    }
    __shared__ double smin[kThreads], smax[kThreads];
    __shared__ long long sidx[kThreads];
    smin[threadIdx.x] = vmin; smax[threadIdx.x] = vmax; sidx[threadIdx.x] = imin;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            const int o = threadIdx.x + s;
            if (smin[o] < smin[threadIdx.x] || (smin[o] == smin[threadIdx.x] && sidx[o] < sidx[threadIdx.x])) {
                smin[threadIdx.x] = smin[o]; sidx[threadIdx.x] = sidx[o];
            }
            if (smax[o] > smax[threadIdx.x]) smax[threadIdx.x] = smax[o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[3 * blockIdx.x + 0] = smin[0];
        part[3 * blockIdx.x + 1] = smax[0];
        part[3 * blockIdx.x + 2] = __longlong_as_double(sidx[0]);
    }
}

__global__ void monopole_final(const double *__restrict__ part, int n, double *__restrict__ out)
{
    if (threadIdx.x != 0) return;
    double vmin = INFINITY, vmax = -INFINITY;
    long long imin = LLONG_MAX;
    for (int i = 0; i < n; ++i) {
        const double a = part[3 * i], c = part[3 * i + 1];
        const long long j = __double_as_longlong(part[3 * i + 2]);
        if (a < vmin || (a == vmin && j < imin)) { vmin = a; imin = j; }
        if (c > vmax) vmax = c;
    }
    out[0] = vmin; out[1] = vmax; out[2] = __longlong_as_double(imin);
}

// ---- truncated model space (Sec. 3.5) ------------------------------------------
// Diagonal element of row r of a block (ascending orbit order, as the oracle
// and the monopole kernel sum it) and its histogram bin, both in FP64.
__device__ __forceinline__ long long trunc_bin(const Blocks &B, const double *__restrict__ d, uint64_t h,
                                               uint32_t l, double lo, double hi, long long bins)
{
    double D = 0.0;
    for (uint32_t w = l; w; w &= w - 1) D += d[__ffs(w) - 1];
    for (uint64_t w = h; w; w &= w - 1) D += d[B.L + __ffsll((long long)w) - 1];
    const long long b = (long long)floor((D - lo) / (hi - lo) * (double)bins);
    return b < bins - 1 ? b : bins - 1;
}

constexpr int kTruncMaxBuckets = 8192;

__global__ void __launch_bounds__(kThreads)
trunc_hist_kernel(const Blocks B, const double *__restrict__ d, double lo, double hi, long long bins,
                  long long lo_bin, int shift, int nbuckets, unsigned long long *__restrict__ hist)
{
    __shared__ unsigned int sh[kTruncMaxBuckets];
    for (int i = threadIdx.x; i < nbuckets; i += blockDim.x) sh[i] = 0u;
    __syncthreads();
    const long long span = (long long)nbuckets << shift;
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        const uint16_t *lw = B.lowword + B.lo_off[k];
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            const long long bin = trunc_bin(B, d, h, lw[r], lo, hi, bins) - lo_bin;
            if (bin >= 0 && bin < span) atomicAdd(&sh[bin >> shift], 1u);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nbuckets; i += blockDim.x)
        if (sh[i]) atomicAdd(hist + i, (unsigned long long)sh[i]);
}

__global__ void __launch_bounds__(kThreads)
trunc_count_kernel(const Blocks B, const double *__restrict__ d, double lo, double hi, long long bins,
                   long long cut, int *__restrict__ blk_kept)
{
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        const uint16_t *lw = B.lowword + B.lo_off[k];
        int cnt = 0;
        for (int r0 = 0; r0 < nk; r0 += kThreads) {
            const int r = r0 + (int)threadIdx.x;
            cnt += __syncthreads_count(r < nk && trunc_bin(B, d, h, lw[r < nk ? r : 0], lo, hi, bins) <= cut);
        }
        if (threadIdx.x == 0) blk_kept[b] = cnt;
    }
}

// kept index = first kept index of the block + rank among the block's kept rows
__global__ void __launch_bounds__(kThreads)
trunc_map_kernel(const Blocks B, const double *__restrict__ d, double lo, double hi, long long bins,
                 long long cut, const int64_t *__restrict__ blk_first, int32_t *__restrict__ map)
{
    __shared__ int swarp[kThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b], base = B.blk_base[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        const uint16_t *lw = B.lowword + B.lo_off[k];
        const int64_t first = blk_first[b];
        int running = 0;
        for (int r0 = 0; r0 < nk; r0 += kThreads) {
            const int r = r0 + (int)threadIdx.x;
            const bool keep = r < nk && trunc_bin(B, d, h, lw[r < nk ? r : 0], lo, hi, bins) <= cut;
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            const int before = __popc(bal & ((1u << lane) - 1u));
            if (lane == 0) swarp[w] = __popc(bal);
            __syncthreads();
            int woff = 0, total = 0;
            for (int i = 0; i < kThreads / 32; ++i) {
                woff += i < w ? swarp[i] : 0;
                total += swarp[i];
            }
            if (r < nk) map[base + r] = keep ? (int32_t)(first + running + woff + before) : -1;
            running += total;
            __syncthreads();
        }
    }
}

// ---- occupation numbers 2 <v| S+_p S-_p |v> ------------------------------------
__global__ void __launch_bounds__(kThreads)
occ_kernel(const Blocks B, const double *__restrict__ v, double *__restrict__ part)
{
    __shared__ double acc[kMaxOmega];
    __shared__ double blk_sum[kThreads];
    for (int p = threadIdx.x; p < B.omega; p += blockDim.x) acc[p] = 0.0;
    __syncthreads();
    for (long long b = blockIdx.x; b < B.nblocks; b += gridDim.x) {
        const uint64_t h = B.blk_h[b], base = B.blk_base[b];
        const int k = B.n - __popcll(h);
        const int nk = (int)B.binom[B.L * kBinomStride + k];
        const uint16_t *lw = B.lowword + B.lo_off[k];
        double mine = 0.0;
        for (int r = threadIdx.x; r < nk; r += blockDim.x) {
            double vr;
            if (B.kept_map) {                     // truncated space: dropped states hold nothing
                const int32_t m = B.kept_map[base + r];
                vr = m >= 0 ? v[m] : 0.0;
            } else {
                vr = v[base + r];
            }
            const double w = vr * vr;
            mine += w;
            for (uint32_t m = lw[r]; m; m &= m - 1) atomicAdd(&acc[__ffs(m) - 1], w);
        }
        blk_sum[threadIdx.x] = mine;
        __syncthreads();
        for (int s = kThreads / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) blk_sum[threadIdx.x] += blk_sum[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0)
            for (uint64_t m = h; m; m &= m - 1) acc[B.L + __ffsll((long long)m) - 1] += blk_sum[0];
        __syncthreads();
    }
    for (int p = threadIdx.x; p < B.omega; p += blockDim.x) part[blockIdx.x * B.omega + p] = acc[p];
}

__global__ void occ_final(const double *__restrict__ part, int n, int omega, double *__restrict__ out)
{
    const int p = threadIdx.x;
    if (p >= omega) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i * omega + p];
    out[p] = 2.0 * s;
}

// ---- float-float rows of an FP32 vector (FP64-accurate, y in FP64) -----------
// Variant 3's kernel with FF coefficients and row sums: x float, y double.
bool ff_fits(const Blocks &B)
{
    return !B.kept_map && layout3<float, FF>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh).total <= kSmemLimit;
}

template <int R>
const void *ff_fn()
{
    return (const void *)hx3_kernel<float, FF, R, false, 4, double>;
}

const void *ff_fn_rows(int rows)
{
    return rows <= 1 ? ff_fn<1>() : rows <= 2 ? ff_fn<2>() : rows <= 4 ? ff_fn<4>() : ff_fn<8>();
}

int grid_ff(const Blocks &B)
{
    const size_t smem = layout3<float, FF>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh).total;
    const void *fn = ff_fn_rows((B.max_block + kThreads - 1) / kThreads);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)sms * per_sm;
    if (g > B.nblocks) g = B.nblocks;
    return (int)(g > 0 ? g : 1);
}

template <int R>
cudaError_t launch_ff_r(const Blocks &B, const FF *G, const FF *d, const float *x, double *y, Tickets *tk,
                        int grid, cudaStream_t st, const int *skip, const HxDot *dot)
{
    const size_t smem = layout3<float, FF>(B.omega, B.L, B.H, B.n, B.max_block, B.max_hh).total;
    cudaError_t err = cudaFuncSetAttribute(ff_fn<R>(), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    hx3_kernel<float, FF, R, false, 4, double><<<grid, kThreads, smem, st>>>(
        B, G, d, x, y, tk, skip, dot ? dot->blk_part : nullptr, dot ? dot->out : nullptr);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_ff(const Blocks &B, const FF *G, const FF *d, const float *x, double *y, Tickets *tk, int grid,
                      cudaStream_t st, const int *skip, const HxDot *dot)
{
    const int rows = (B.max_block + kThreads - 1) / kThreads;
    if (rows <= 1) return launch_ff_r<1>(B, G, d, x, y, tk, grid, st, skip, dot);
    if (rows <= 2) return launch_ff_r<2>(B, G, d, x, y, tk, grid, st, skip, dot);
    if (rows <= 4) return launch_ff_r<4>(B, G, d, x, y, tk, grid, st, skip, dot);
    return launch_ff_r<8>(B, G, d, x, y, tk, grid, st, skip, dot);
}

}  // namespace

size_t hx_smem_bytes(const Blocks &B, int precision)
{
    return precision == 0 ? kernel_smem<double, double>(B) : kernel_smem<float, float>(B);
}

int hx_variant(const Blocks &B, int precision)
{
    if (precision == 0 ? use_v3<double, double>(B) : use_v3<float, float>(B)) return B.variant;
    return (precision == 0 ? use_v2<double, double>(B) : use_v2<float, float>(B)) ? 2 : 1;
}

int hx_grid(const Blocks &B, int precision)
{
    if (precision == 2) return ff_fits(B) ? grid_ff(B) : 0;
    return precision == 0 ? grid_prec<double, double>(B) : grid_prec<float, float>(B);
}

cudaError_t hx_launch(const Blocks &B, const HxProblem &P, int precision, const void *x, void *y,
                      Tickets *tk, int grid, cudaStream_t st, const int *skip, const HxDot *dot)
{
    if (dot && (!dot->blk_part || !dot->out)) return cudaErrorInvalidValue;
    if (precision == 2) {
        if (!ff_fits(B) || !P.Gff || !P.dff || grid < 1) return cudaErrorNotSupported;
        return launch_ff(B, reinterpret_cast<const FF *>(P.Gff), reinterpret_cast<const FF *>(P.dff),
                         static_cast<const float *>(x), static_cast<double *>(y), tk, grid, st, skip, dot);
    }
    if (precision == 0) return launch_prec<double, double>(B, P.G64, P.d64, x, y, tk, grid, st, skip, dot);
    return launch_prec<float, float>(B, P.G32, P.d32, x, y, tk, grid, st, skip, dot);
}

namespace {
// the batched variant-3 kernel when asked for and its shared memory fits
template <typename T, typename A>
bool batch_v3(const BatchBlocks &BB)
{
    return BB.variant == 3 &&
           layout3<T, A>(BB.max_omega, BB.max_L, BB.max_H, BB.max_n, BB.max_block, BB.max_hh).total <= kSmemLimit;
}

template <typename T, typename A, int R>
const void *batch_fn(bool v3)
{
    return v3 ? (const void *)hx3_batch_kernel<T, A, R> : (const void *)hx_batch_kernel<T, A, R>;
}

template <typename T, typename A>
const void *batch_fn_rows(int rows, bool v3)
{
    return rows <= 1 ? batch_fn<T, A, 1>(v3) : rows <= 2 ? batch_fn<T, A, 2>(v3) : rows <= 4 ? batch_fn<T, A, 4>(v3)
                                                                                            : batch_fn<T, A, 8>(v3);
}

template <typename T, typename A>
size_t batch_smem(const BatchBlocks &BB)
{
    return batch_v3<T, A>(BB)
               ? layout3<T, A>(BB.max_omega, BB.max_L, BB.max_H, BB.max_n, BB.max_block, BB.max_hh).total
               : layout<T, A>(BB.max_omega, BB.max_L, BB.max_H, BB.max_block, BB.max_hh).total;
}

template <typename T, typename A>
cudaError_t batch_launch_t(const BatchBlocks &BB, const A *G, const A *d, const void *x, void *y,
                           unsigned long long *counter, int grid, cudaStream_t st, const int *skip,
                           int skip_stride)
{
    const bool v3 = batch_v3<T, A>(BB);
    const size_t smem = batch_smem<T, A>(BB);
    const int rows = (BB.max_block + kThreads - 1) / kThreads;
    cudaError_t err = cudaFuncSetAttribute(batch_fn_rows<T, A>(rows, v3),
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    const T *xt = static_cast<const T *>(x);
    T *yt = static_cast<T *>(y);
    if (v3) {
        if (rows <= 1) hx3_batch_kernel<T, A, 1><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
        else if (rows <= 2) hx3_batch_kernel<T, A, 2><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
        else if (rows <= 4) hx3_batch_kernel<T, A, 4><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
        else hx3_batch_kernel<T, A, 8><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
        count_launches(1);
        return cudaGetLastError();
    }
    if (rows <= 1) hx_batch_kernel<T, A, 1><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
    else if (rows <= 2) hx_batch_kernel<T, A, 2><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
    else if (rows <= 4) hx_batch_kernel<T, A, 4><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
    else hx_batch_kernel<T, A, 8><<<grid, kThreads, smem, st>>>(BB, G, d, xt, yt, counter, skip, skip_stride);
    count_launches(1);
    return cudaGetLastError();
}

template <typename T, typename A>
int batch_grid_t(const BatchBlocks &BB)
{
    const size_t smem = batch_smem<T, A>(BB);
    const void *fn = batch_fn_rows<T, A>((BB.max_block + kThreads - 1) / kThreads, batch_v3<T, A>(BB));
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)sms * per_sm;
    if (g > BB.nblocks) g = BB.nblocks;
    return (int)(g > 0 ? g : 1);
}

// Batched float-float rows of FP32 vectors (x float, y double): the batched
// variant-3 kernel with FF coefficients, where its shared memory fits
bool batch_ff_fits(const BatchBlocks &BB)
{
    return layout3<float, FF>(BB.max_omega, BB.max_L, BB.max_H, BB.max_n, BB.max_block, BB.max_hh).total <=
           kSmemLimit;
}

template <int R>
const void *batch_ff_fn()
{
    return (const void *)hx3_batch_kernel<float, FF, R, double>;
}

const void *batch_ff_fn_rows(int rows)
{
    return rows <= 1 ? batch_ff_fn<1>() : rows <= 2 ? batch_ff_fn<2>() : rows <= 4 ? batch_ff_fn<4>() : batch_ff_fn<8>();
}

cudaError_t batch_launch_ff(const BatchBlocks &BB, const FF *G, const FF *d, const float *x, double *y,
                            unsigned long long *counter, int grid, cudaStream_t st, const int *skip, int skip_stride)
{
    const size_t smem = layout3<float, FF>(BB.max_omega, BB.max_L, BB.max_H, BB.max_n, BB.max_block, BB.max_hh).total;
    const int rows = (BB.max_block + kThreads - 1) / kThreads;
    cudaError_t err = cudaFuncSetAttribute(batch_ff_fn_rows(rows), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem);
    if (err != cudaSuccess) return err;
    if (rows <= 1) hx3_batch_kernel<float, FF, 1, double><<<grid, kThreads, smem, st>>>(BB, G, d, x, y, counter, skip, skip_stride);
    else if (rows <= 2) hx3_batch_kernel<float, FF, 2, double><<<grid, kThreads, smem, st>>>(BB, G, d, x, y, counter, skip, skip_stride);
    else if (rows <= 4) hx3_batch_kernel<float, FF, 4, double><<<grid, kThreads, smem, st>>>(BB, G, d, x, y, counter, skip, skip_stride);
    else hx3_batch_kernel<float, FF, 8, double><<<grid, kThreads, smem, st>>>(BB, G, d, x, y, counter, skip, skip_stride);
    count_launches(1);
    return cudaGetLastError();
}

int batch_grid_ff(const BatchBlocks &BB)
{
    const size_t smem = layout3<float, FF>(BB.max_omega, BB.max_L, BB.max_H, BB.max_n, BB.max_block, BB.max_hh).total;
    const void *fn = batch_ff_fn_rows((BB.max_block + kThreads - 1) / kThreads);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    int64_t g = (int64_t)sms * per_sm;
    if (g > BB.nblocks) g = BB.nblocks;
    return (int)(g > 0 ? g : 1);
}
}  // namespace

cudaError_t hx_batch_launch(const BatchBlocks &BB, const HxProblem &P, int precision, const void *x, void *y,
                            unsigned long long *counter, int grid, cudaStream_t st, const int *skip, int skip_stride)
{
    unsigned long long *ctr = counter;
    if (precision == 2) {
        if (!batch_ff_fits(BB) || !P.Gff || !P.dff || grid < 1) return cudaErrorNotSupported;
        return batch_launch_ff(BB, reinterpret_cast<const FF *>(P.Gff), reinterpret_cast<const FF *>(P.dff),
                               static_cast<const float *>(x), static_cast<double *>(y), ctr, grid, st, skip,
                               skip_stride);
    }
    if (precision == 0) return batch_launch_t<double, double>(BB, P.G64, P.d64, x, y, ctr, grid, st, skip, skip_stride);
    return batch_launch_t<float, float>(BB, P.G32, P.d32, x, y, ctr, grid, st, skip, skip_stride);
}

int hx_batch_grid(const BatchBlocks &BB, int precision)
{
    if (precision == 2) return batch_ff_fits(BB) ? batch_grid_ff(BB) : 0;
    return precision == 0 ? batch_grid_t<double, double>(BB) : batch_grid_t<float, float>(BB);
}

cudaError_t monopole_launch(const Blocks &B, const double *d64, double *partials, int grid,
                            double *out, cudaStream_t st)
{
    monopole_kernel<<<grid, kThreads, 0, st>>>(B, d64, partials);
    monopole_final<<<1, 32, 0, st>>>(partials, grid, out);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t trunc_hist_launch(const Blocks &B, const double *d64, double lo, double hi, int64_t bins,
                              int64_t lo_bin, int shift, int nbuckets, unsigned long long *hist, int grid,
                              cudaStream_t st)
{
    if (nbuckets < 1 || nbuckets > kTruncMaxBuckets) return cudaErrorInvalidValue;
    trunc_hist_kernel<<<grid, kThreads, 0, st>>>(B, d64, lo, hi, bins, lo_bin, shift, nbuckets, hist);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t trunc_count_launch(const Blocks &B, const double *d64, double lo, double hi, int64_t bins,
                               int64_t cut, int *blk_kept, int grid, cudaStream_t st)
{
    trunc_count_kernel<<<grid, kThreads, 0, st>>>(B, d64, lo, hi, bins, cut, blk_kept);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t trunc_map_launch(const Blocks &B, const double *d64, double lo, double hi, int64_t bins,
                             int64_t cut, const int64_t *blk_first, int32_t *map, int grid, cudaStream_t st)
{
    trunc_map_kernel<<<grid, kThreads, 0, st>>>(B, d64, lo, hi, bins, cut, blk_first, map);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t occupations_launch(const Blocks &B, const double *v, double *partials, int grid,
                               double *out, cudaStream_t st)
{
    occ_kernel<<<grid, kThreads, 0, st>>>(B, v, partials);
    occ_final<<<1, 64, 0, st>>>(partials, grid, B.omega, out);
    count_launches(2);
    return cudaGetLastError();
}

}  // namespace pd
