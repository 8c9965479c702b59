// pd_api.cu -- the C ABI (include/pairdiag.h): handle creation (block tables
// of the basis), H*x entry points and the restarted-Lanczos driver.
//
// The driver follows Algorithm 2 of the paper with full reorthogonalisation
// (classical Gram-Schmidt applied twice against every stored Lanczos vector),
// the tridiagonal eigenproblem of each cycle solved on the device, and restart
// from the ground Ritz vector (Sec. 3.4).  Convergence is the paper's
// |beta_1/alpha_1| <= tol measured at the first step of each cycle (Sec. 5.1).
#include "pd_internal.h"
#include "pairdiag.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

using namespace pd;

namespace pd {
std::atomic<long long> g_kernel_launches{0};
}

namespace {
thread_local std::string g_last_error = "no error";

// autotuned H*x schedules: (omega, n, precision) -> (low_bits, hx_variant)
struct TuneKey {
    int omega, n, precision;
    bool operator<(const TuneKey &o) const
    {
        return omega != o.omega ? omega < o.omega : n != o.n ? n < o.n : precision < o.precision;
    }
};
std::mutex g_tune_mutex;
std::map<TuneKey, std::pair<int, int>> g_tune;

// Largest-first block order for the full-space H*x: built for at most
// kLptMaxBlocks blocks, used while a launch has at most kLptPerCta blocks per
// CTA (beyond that the tail of one block is a small part of a launch, and the
// ascending order keeps concurrently processed blocks close in the basis)
constexpr int64_t kLptMaxBlocks = (int64_t)1 << 18;
constexpr int64_t kLptPerCta = 64;

bool tuned_schedule(int omega, int n, int precision, int *low_bits, int *variant)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(TuneKey{omega, n, precision});
    if (it == g_tune.end()) return false;
    *low_bits = it->second.first;
    *variant = it->second.second;
    return true;
}
}

namespace pd {

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int sm_count()
{
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        dev = -1;
    }
    if (dev >= 0) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0) return c;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev < 0 ? 0 : dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    if (dev >= 0) cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

uint64_t host_binom(int n, int m)
{
    static uint64_t table[64][64];
    static bool ready = false;
    if (!ready) {
        memset(table, 0, sizeof table);
        for (int i = 0; i < 64; ++i) {
            table[i][0] = 1;
            for (int j = 1; j <= i; ++j) table[i][j] = table[i - 1][j - 1] + table[i - 1][j];
        }
        ready = true;
    }
    if (n < 0 || m < 0 || m > n || n > 63) return 0;
    return table[n][m];
}

// words of `bits` bits with `c` set bits, ascending (Gosper's successor)
void words_with_popcount(int bits, int c, std::vector<uint64_t> &out)
{
    if (c == 0) { out.push_back(0); return; }
    if (c > bits) return;
    uint64_t w = (c == 64) ? ~0ull : ((1ull << c) - 1ull);
    const uint64_t last = w << (bits - c);
    for (;;) {
        out.push_back(w);
        if (w == last) break;
        const uint64_t lowest = w & (~w + 1ull);
        const uint64_t ripple = w + lowest;
        w = ripple | (((w ^ ripple) >> 2) / lowest);
    }
}

uint64_t host_block_base(uint64_t hw, int L, int N)
{
    int ord = N - __builtin_popcountll(hw);
    uint64_t s = 0;
    for (int p = 0; p < 64; ++p)
        if (hw >> p & 1ull) s += host_binom(L + p, ++ord);
    return s;
}

}  // namespace pd

struct pairdiag {
    int omega = 0, n = 0;
    pairdiag_options opt{};
    std::vector<double> e, G, d;
    int64_t dim = 0, nnz = 0;        // of the space the solver works in (kept states when truncated)
    int64_t full_dim = 0, full_nnz = 0;   // C(Omega, N) and its off-diagonal nonzeros
    int32_t *d_kmap = nullptr;       // truncated space (Sec. 3.5): full index -> kept index, -1 dropped
    uint64_t *d_kblk_h = nullptr, *d_kblk_base = nullptr;   // the blocks holding kept states
    // the block list in the order the persistent H*x kernels take it when
    // there are few blocks per CTA: largest blocks first (ascending high word
    // within a size), so the launch does not end on one CTA's large block
    uint64_t *d_lpt_h = nullptr, *d_lpt_base = nullptr;
    Blocks B{};
    int device = 0;
    cudaStream_t st = nullptr;
    // tables
    uint64_t *d_blk_h = nullptr, *d_blk_base = nullptr, *d_binom = nullptr;
    uint16_t *d_lowword = nullptr, *d_rankL = nullptr;
    double *d_G64 = nullptr, *d_d64 = nullptr;
    float *d_G32 = nullptr, *d_d32 = nullptr;
    float2 *d_Gff = nullptr, *d_dff = nullptr;   // G and d split into two FP32 parts (float-float rows)
    Tickets *d_tk = nullptr;         // counters of the persistent and streaming kernels
    double *d_blkdot = nullptr;      // [nblocks] per-block partial sums of the fused alpha
    double *d_part = nullptr;        // partial sums of the streaming kernels
    size_t part_count = 0;
    LanczosScalars *d_S = nullptr;
    double *d_small = nullptr;       // [8] small outputs
    int hxgrid[3] = {0, 0, 0};       // per H*x precision (2: float-float rows; 0 = not available)
    int rgrid = 0;                   // grid of the per-row reductions
    // Lanczos window (lazily allocated) per storage type
    void *d_Q[2] = {nullptr, nullptr};
    int64_t ldq = 0;                 // stride between window vectors: dim rounded up to 4 elements
    int Qwin[2] = {0, 0};
    void *d_p[2] = {nullptr, nullptr};
    double *d_v64 = nullptr, *d_w64 = nullptr;
    std::vector<double> start;
    std::vector<double> start_w;     // per-orbit weights of a product start vector
    // converged eigenvectors locked out of the Krylov space (lowest few states):
    // while n_locked > 0 every H*x result and restart vector is projected
    // against them
    int n_locked = 0;
    int lock_cap = 0;
    double *d_L64 = nullptr;         // [lock_cap * ldq] FP64 locked vectors
    float *d_L32 = nullptr;          // their FP32 copies (mixed form)
    double *d_lockc = nullptr;       // [kMaxWindow] projection coefficients
    pairdiag_mlp *mlp = nullptr;     // network predicting them (PD_START_MLP)
    // the fused Lanczos step (one cooperative launch per step) per storage type;
    // planned for the window buffer step_q[dtype]
    bool step_fusion = true;
    StepPlan step[2];
    const void *step_q[2] = {nullptr, nullptr};
    // optional event timing of H*x launches
    bool profiling = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> hx_events;
    std::vector<int> hx_event_prec;
    size_t hx_events_used = 0;
};

namespace {

void free_all(pairdiag *h)
{
    for (auto &ev : h->hx_events) {
        cudaEventDestroy(ev.first);
        cudaEventDestroy(ev.second);
    }
    h->hx_events.clear();
    void *ptrs[] = {h->d_blk_h, h->d_blk_base, h->d_binom, h->d_lowword, h->d_rankL, h->d_G64,
                    h->d_d64, h->d_G32, h->d_d32, h->d_tk, h->d_blkdot, h->d_part, h->d_S, h->d_small,
                    h->d_Q[0], h->d_Q[1], h->d_p[0], h->d_p[1], h->d_v64, h->d_w64,
                    h->d_L64, h->d_L32, h->d_lockc, h->d_kmap, h->d_kblk_h, h->d_kblk_base,
                    h->d_lpt_h, h->d_lpt_base, h->d_Gff, h->d_dff};
    // the blocks go back to the library's cache: no queued kernel may still use
    // them.  Every kernel and copy of the handle runs on its stream, so that
    // stream's completion is enough (other streams of the caller go on).
    cudaStreamSynchronize(h->st);
    for (void *p : ptrs) pool_free(p);
}

template <typename T>
int dalloc(T **p, size_t count)
{
    void *q = nullptr;
    cudaError_t e = pool_alloc(&q, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA, "cudaMalloc(%zu bytes): %s",
                    count * sizeof(T), cudaGetErrorString(e));
    }
    *p = static_cast<T *>(q);
    return PD_OK;
}

template <typename T>
int upload(T **p, const std::vector<T> &v)
{
    PD_TRY(dalloc(p, v.size()));
    PD_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return PD_OK;
}

int build_tables(pairdiag *h)
{
    const int omega = h->omega, N = h->n;
    int L = h->opt.low_bits > 0 ? h->opt.low_bits : 12;
    L = std::min(L, std::min(omega, kMaxLow));
    const int H = omega - L;
    // admissible k (pairs in the low orbits)
    const int kmin = std::max(0, N - H), kmax = std::min(N, L);
    int64_t nblocks = 0;
    int max_block = 0, max_hh = 0, max_stage = 0;
    for (int k = kmin; k <= kmax; ++k) {
        const int ph = N - k;
        nblocks += (int64_t)host_binom(H, ph);
        max_block = std::max(max_block, (int)host_binom(L, k));
        max_hh = std::max(max_hh, ph * (H - ph));
        const int64_t up = (k < L && ph > 0) ? ph * (int64_t)host_binom(L, k + 1) : 0;
        const int64_t dn = (k > 0 && H - ph > 0) ? (H - ph) * (int64_t)host_binom(L, k - 1) : 0;
        max_stage = (int)std::max<int64_t>(max_stage, up + dn);
    }
    // the persistent H*x kernels keep block indices in int, and their counters
    // run past nblocks by up to two per CTA before every CTA has stopped
    if (nblocks > (int64_t)INT_MAX - (int64_t)(1 << 20))
        return fail(PD_ENOTSUP, "too many basis blocks (%lld)", (long long)nblocks);
    std::vector<uint64_t> hw;
    hw.reserve((size_t)nblocks);
    for (int k = kmin; k <= kmax; ++k) words_with_popcount(H, N - k, hw);
    std::sort(hw.begin(), hw.end());
    std::vector<uint64_t> base(hw.size());
    uint64_t run = 0;
    for (size_t b = 0; b < hw.size(); ++b) {
        base[b] = host_block_base(hw[b], L, N);
        if (base[b] != run) return fail(PD_ECUDA, "internal: block index mismatch at block %zu", b);
        run += host_binom(L, N - __builtin_popcountll(hw[b]));
    }
    if ((int64_t)run != h->full_dim) return fail(PD_ECUDA, "internal: blocks cover %llu of %lld states",
                                                 (unsigned long long)run, (long long)h->full_dim);
    // low-word tables
    const int nL = 1 << L;
    std::vector<uint16_t> lowword(nL), rankL(nL);
    std::vector<int> fill(L + 2, 0);
    int off[kMaxLow + 2];
    off[0] = 0;
    for (int k = 0; k <= L; ++k) off[k + 1] = off[k] + (int)host_binom(L, k);
    for (int w = 0; w < nL; ++w) {
        const int k = __builtin_popcount(w);
        rankL[w] = (uint16_t)fill[k];
        lowword[off[k] + fill[k]] = (uint16_t)w;
        ++fill[k];
    }
    std::vector<uint64_t> binom(64 * 64);
    for (int i = 0; i < 64; ++i)
        for (int j = 0; j < 64; ++j) binom[i * 64 + j] = host_binom(i, j);

    PD_TRY(upload(&h->d_blk_h, hw));
    PD_TRY(upload(&h->d_blk_base, base));
    if ((int64_t)hw.size() <= kLptMaxBlocks) {
        std::vector<uint32_t> order(hw.size());
        for (size_t b = 0; b < order.size(); ++b) order[b] = (uint32_t)b;
        auto rows = [&](uint32_t b) { return host_binom(L, N - __builtin_popcountll(hw[b])); };
        std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return rows(a) > rows(b); });
        std::vector<uint64_t> lh(hw.size()), lb(hw.size());
        for (size_t b = 0; b < order.size(); ++b) {
            lh[b] = hw[order[b]];
            lb[b] = base[order[b]];
        }
        PD_TRY(upload(&h->d_lpt_h, lh));
        PD_TRY(upload(&h->d_lpt_base, lb));
    }
    PD_TRY(upload(&h->d_lowword, lowword));
    PD_TRY(upload(&h->d_rankL, rankL));
    PD_TRY(upload(&h->d_binom, binom));

    Blocks &B = h->B;
    B.omega = omega; B.n = N; B.L = L; B.H = H;
    B.nblocks = (int64_t)hw.size();
    B.max_block = max_block;
    B.max_hh = max_hh;
    B.max_stage = max_stage;
    B.variant = h->opt.hx_variant;
    B.blk_h = h->d_blk_h; B.blk_base = h->d_blk_base;
    B.lowword = h->d_lowword; B.rankL = h->d_rankL; B.binom = h->d_binom;
    for (int k = 0; k <= kMaxLow + 1; ++k) B.lo_off[k] = (k <= L + 1) ? off[k] : off[L + 1];
    return PD_OK;
}

int ensure_window(pairdiag *h, int dtype, int window)
{
    const size_t es = dtype == 0 ? sizeof(double) : sizeof(float);
    if (h->d_Q[dtype] && h->Qwin[dtype] >= window) return PD_OK;
    if (h->d_Q[dtype]) {                          // a larger window: the old one may still be in use
        cudaStreamSynchronize(h->st);
        pool_free(h->d_Q[dtype]);
        h->d_Q[dtype] = nullptr;
    }
    void *q = nullptr;
    cudaError_t e = pool_alloc(&q, es * (size_t)window * (size_t)h->ldq);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(PD_ENOMEM, "Lanczos window of %d x %lld elements: %s", window, (long long)h->dim,
                    cudaGetErrorString(e));
    }
    h->d_Q[dtype] = q;
    h->Qwin[dtype] = window;
    if (!h->d_p[dtype]) {
        e = pool_alloc(&h->d_p[dtype], es * (size_t)h->dim);
        if (e != cudaSuccess) { cudaGetLastError(); return fail(PD_ENOMEM, "work vector: %s", cudaGetErrorString(e)); }
    }
    return PD_OK;
}

int ensure_fp64_pair(pairdiag *h)
{
    if (!h->d_v64) PD_TRY(dalloc(&h->d_v64, (size_t)h->dim));
    if (!h->d_w64) PD_TRY(dalloc(&h->d_w64, (size_t)h->dim));
    return PD_OK;
}

// While profiling: a pair of events for one timed region of record kind
// `code` (0/1: an H*x launch of that precision; 2 + dtype: the vector work of
// one Lanczos step), its start recorded on the handle's stream; else nullptr
int prof_begin(pairdiag *h, int code, std::pair<cudaEvent_t, cudaEvent_t> **ev)
{
    *ev = nullptr;
    if (!h->profiling) return PD_OK;
    if (h->hx_events_used == h->hx_events.size()) {
        std::pair<cudaEvent_t, cudaEvent_t> e2;
        PD_CUDA(cudaEventCreate(&e2.first));
        PD_CUDA(cudaEventCreate(&e2.second));
        h->hx_events.push_back(e2);
        h->hx_event_prec.push_back(0);
    }
    h->hx_event_prec[h->hx_events_used] = code;
    *ev = &h->hx_events[h->hx_events_used++];
    PD_CUDA(cudaEventRecord((*ev)->first, h->st));
    return PD_OK;
}

// y = H x; with dot_out also x^T y -> *dot_out (fused into the same launch)
int hx(pairdiag *h, int precision, const void *x, void *y, const int *skip = nullptr, double *dot_out = nullptr)
{
    HxProblem P{h->d_G64, h->d_d64, h->d_G32, h->d_d32, h->d_Gff, h->d_dff};
    std::pair<cudaEvent_t, cudaEvent_t> *ev = nullptr;
    PD_TRY(prof_begin(h, precision == 2 ? 0 : precision, &ev));    // float-float rows count as FP64
    const HxDot dot{h->d_blkdot, dot_out};
    Blocks B = h->B;
    if (h->d_lpt_h && !B.kept_map && B.nblocks <= kLptPerCta * (int64_t)h->hxgrid[precision]) {
        B.blk_h = h->d_lpt_h;
        B.blk_base = h->d_lpt_base;
    }
    PD_CUDA(hx_launch(B, P, precision, x, y, h->d_tk, h->hxgrid[precision], h->st, skip,
                      dot_out ? &dot : nullptr));
    if (ev) PD_CUDA(cudaEventRecord(ev->second, h->st));
    return PD_OK;
}

template <typename T>
T *vec(void *base, int64_t i, int64_t dim) { return static_cast<T *>(base) + i * dim; }

// device scratch for the 2^L low-word factors of a product start vector
double *factor_scratch(pairdiag *h)
{
    return h->part_count >= ((size_t)1 << h->B.L) ? h->d_part : nullptr;
}

void *qvec(pairdiag *h, int dtype, int i)
{
    const size_t es = dtype == 0 ? 8 : 4;
    return static_cast<char *>(h->d_Q[dtype]) + es * (size_t)i * (size_t)h->ldq;
}

// v <- v - L (L^T v) against the locked vectors L (storage type dtype): the
// projected operator whose lowest eigenpair is the next state
int lock_project(pairdiag *h, int dtype, void *v, const int *skip)
{
    if (h->n_locked == 0) return PD_OK;
    const void *L = dtype == 0 ? static_cast<const void *>(h->d_L64) : static_cast<const void *>(h->d_L32);
    PD_CUDA(multidot_launch(dtype, L, h->ldq, h->n_locked, v, h->dim, h->d_part, h->d_lockc, h->st, skip,
                            &h->d_tk->vec_done));
    PD_CUDA(update_launch(dtype, L, h->ldq, h->n_locked, h->d_lockc, v, h->dim, h->d_part, nullptr, h->st, skip));
    return PD_OK;
}

// err: the barrier error flag, copied back with the cycle's scalars.
// PD_ETIMEOUT (and the barrier state reset) when a grid-wide wait of a fused
// step gave up.
int check_barrier(pairdiag *h, int err)
{
    if (!err) return PD_OK;
    PD_CUDA(cudaMemsetAsync(&h->d_tk->bar, 0, sizeof(GridBar), h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    return fail(PD_ETIMEOUT, "a grid-wide barrier of the fused Lanczos step timed out");
}

struct CycleStats {
    int iterations = 0;
    int restarts = 0;
    double rel = INFINITY;       // |beta_1/alpha_1| of the last restart vector
    double energy = 0.0;         // Rayleigh quotient (converged) or last Ritz value
    double gap = INFINITY;
    bool converged = false;
};

// The fused step's plan for the current window buffer of dtype; false where
// the three-kernel form runs instead
bool fused_step(pairdiag *h, int dtype)
{
    if (!h->step_fusion) return false;
    if (h->step_q[dtype] != h->d_Q[dtype]) {
        h->step[dtype] = StepPlan{};
        step_plan(dtype, h->dim, h->ldq, h->d_Q[dtype], h->d_p[dtype], &h->step[dtype]);
        h->step_q[dtype] = h->d_Q[dtype];
    }
    return h->step[dtype].grid > 0;
}

// One Lanczos step i of a cycle of m on storage type dtype (Algorithm 2 with
// full reorthogonalisation, Sec. 3.4):
//   1. p = H q_i and alpha = q_i^T p (the dot fused into the H*x launch);
//   2. the three-term recurrence p -= alpha q_i + beta_{i-1} q_{i-1} with the
//      projections c = Q^T p of one Gram-Schmidt pass against every stored
//      vector;
//   3. p -= Q c with ||p||^2, then alpha_i = alpha + c_i, beta_i = ||p||;
//   4. q_{i+1} = p / beta_i (i + 1 < m).
// The recurrence followed by the full pass is Gram-Schmidt applied twice.
// Fused form: 2-4 are one cooperative launch with grid-wide barriers.  Else
// 2 and 3 are two launches whose sums are finished by their last CTA, and 4
// is the scaling at the start of the next step.  Every kernel is skipped once
// S->broken is set (breakdown or a converged Ritz estimate earlier in the cycle).
int lanczos_step(pairdiag *h, int dtype, int i, int m)
{
    const int64_t dim = h->dim;
    LanczosScalars *S = h->d_S;
    const int *skip = &S->broken;
    void *Q = h->d_Q[dtype];
    void *p = h->d_p[dtype];
    cudaStream_t st = h->st;
    const int64_t ld = h->ldq;
    unsigned long long *tk = &h->d_tk->vec_done;
    PD_TRY(hx(h, dtype, qvec(h, dtype, i), p, skip, S->c1));
    std::pair<cudaEvent_t, cudaEvent_t> *ev = nullptr;
    PD_TRY(prof_begin(h, 2 + dtype, &ev));
    if (h->n_locked) PD_TRY(lock_project(h, dtype, p, skip));
    if (fused_step(h, dtype)) {
        PD_CUDA(step_launch(dtype, h->step[dtype], Q, ld, i, S, p, dim, h->d_part, &h->d_tk->bar,
                            i + 1 < m ? qvec(h, dtype, i + 1) : nullptr, st));
    } else {
        PD_CUDA(recur_project_launch(dtype, Q, ld, i, S, p, dim, h->d_part, S->c2, st, skip, tk));
        PD_CUDA(update_launch(dtype, Q, ld, i + 1, S->c2, p, dim, h->d_part, &S->norm2, st, skip, tk, S, i));
    }
    if (ev) PD_CUDA(cudaEventRecord(ev->second, st));
    return PD_OK;
}

// Restarted Lanczos on storage type dtype.  Q_0 holds the start vector (any
// norm).  On return Q_0 is the normalised best vector.  The host synchronises
// once per cycle (to test convergence on the restart vector); breakdown inside
// a cycle is handled on the device.
// Lanczos steps between two estimates of the cycle's Ritz residual
constexpr int kRitzCheckEvery = 4;

int run_cycles(pairdiag *h, int dtype, double tol, int max_cycles, CycleStats &cs)
{
    const int64_t dim = h->dim;
    const int m = (int)std::min<int64_t>(std::max(1, h->opt.window), std::min<int64_t>(dim, kMaxWindow));
    cudaStream_t st = h->st;
    LanczosScalars *S = h->d_S;
    void *Q = h->d_Q[dtype];
    void *p = h->d_p[dtype];
    const int *skip = &S->broken;
    // normalise the start vector
    unsigned long long *tk = &h->d_tk->vec_done;
    PD_CUDA(multidot_launch(dtype, Q, h->ldq, 1, Q, dim, h->d_part, &S->dots[0], st, nullptr, tk));
    PD_CUDA(scale_launch(dtype, Q, Q, dim, &S->dots[0], 1, st));
    std::vector<double> history;                  // |beta_1/alpha_1| per cycle
    bool ended_early = false;                     // the last cycle stopped before the full window
    double est_tol = tol;                         // threshold of the Ritz estimate
    // One synchronisation per cycle: the end of a cycle (its Ritz values) and
    // step 0 of the next (the restart test) are read back together.
    double ab[2] = {0.0, 0.0}, th[2] = {0.0, 0.0};
    int used = 0, berr = 0;
    auto begin_cycle = [&]() -> int {
        if (h->n_locked) {                        // restart vector orthogonal to the locked states
            PD_TRY(lock_project(h, dtype, Q, nullptr));
            PD_CUDA(multidot_launch(dtype, Q, h->ldq, 1, Q, dim, h->d_part, &S->dots[0], st, nullptr, tk));
            PD_CUDA(scale_launch(dtype, Q, Q, dim, &S->dots[0], 1, st));
        }
        PD_CUDA(cycle_reset_launch(S, st));
        PD_TRY(lanczos_step(h, dtype, 0, m));
        PD_CUDA(cudaMemcpyAsync(&ab[0], &S->alpha[0], sizeof(double), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaMemcpyAsync(&ab[1], &S->beta[0], sizeof(double), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaMemcpyAsync(&berr, &h->d_tk->bar.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        return PD_OK;
    };
    auto end_cycle = [&](int cycle) -> int {     // after the synchronisation
        cs.iterations += used - 1;
        ended_early = used < m;
        if (!std::isfinite(th[0])) return fail(PD_ECUDA, "non-finite Ritz value in cycle %d", cycle);
        cs.energy = th[0];
        cs.gap = th[1] - th[0];
        return PD_OK;
    };
    PD_TRY(begin_cycle());
    bool pending = false;                         // the previous cycle's end is still to be read
    for (int cycle = 0; cycle <= max_cycles; ++cycle) {
        PD_CUDA(cudaStreamSynchronize(st));
        PD_TRY(check_barrier(h, berr));
        if (pending) {
            PD_TRY(end_cycle(cycle - 1));
            ++cs.restarts;
            pending = false;
        }
        ++cs.iterations;
        if (!std::isfinite(ab[0]) || !std::isfinite(ab[1]))
            return fail(PD_ECUDA, "non-finite Lanczos coefficient in cycle %d", cycle);
        cs.rel = (ab[1] == 0.0) ? 0.0 : ab[1] / std::fabs(ab[0]);
        cs.energy = ab[0];
        if (h->opt.mode == 0) {
            if (cs.rel <= tol) {
                cs.converged = true;
                return PD_OK;
            }
            // FP32 vectors: stop once the residual no longer falls (rounding floor);
            // the caller refines in FP64
            history.push_back(cs.rel);
            const size_t nh = history.size();
            if (dtype == 1 && nh >= 4 && fp32_stalled(history[nh - 1], history[nh - 4], tol)) return PD_OK;
        }
        // the Ritz estimate stopped the last cycle early but the restart test
        // failed (the estimate was optimistic, e.g. near the rounding floor of
        // the vectors): later cycles stop only at a 4x smaller estimate
        if (ended_early) est_tol *= 0.25;
        const bool fused = fused_step(h, dtype);
        for (int i = 1; i < m; ++i) {
            if (!fused) PD_CUDA(scale_launch(dtype, p, qvec(h, dtype, i), dim, &S->beta[i - 1], 0, st, skip));
            PD_TRY(lanczos_step(h, dtype, i, m));
            // restarted mode: end the cycle as soon as its lowest Ritz pair is
            // converged, instead of running the whole window
            if (h->opt.mode == 0 && (i + 1) % kRitzCheckEvery == 0 && i + 1 < m)
                PD_CUDA(ritz_estimate_launch(S, i, est_tol, st));
        }
        PD_CUDA(tridiag_launch(S, 0, st));
        PD_CUDA(ritz_launch(dtype, Q, h->ldq, &S->used, S->s, dim, h->d_part, &S->norm2, st, tk));
        PD_CUDA(scale_launch(dtype, Q, Q, dim, &S->norm2, 1, st));
        PD_CUDA(cudaMemcpyAsync(th, S->theta, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaMemcpyAsync(&used, &S->used, sizeof(int), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaMemcpyAsync(&berr, &h->d_tk->bar.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (h->opt.mode == 1 || cycle == max_cycles) {   // no next cycle
            PD_CUDA(cudaStreamSynchronize(st));
            PD_TRY(check_barrier(h, berr));
            PD_TRY(end_cycle(cycle));
            if (h->opt.mode == 1) cs.converged = true;
            return PD_OK;
        }
        pending = true;
        PD_TRY(begin_cycle());                    // step 0 of the next cycle from the restart vector
    }
    return PD_OK;
}

int init_start(pairdiag *h, int dtype)
{
    void *q0 = qvec(h, dtype, 0);
    const int64_t dim = h->dim;
    switch (h->opt.start) {
    case PD_START_RANDOM:
        PD_CUDA(random_start_launch(dtype, q0, dim, h->opt.seed, h->st));
        break;
    case PD_START_FIRST:
    case PD_START_HF: {
        int64_t pos = 0;
        if (h->opt.start == PD_START_HF) {
            double dmin, dmax;
            PD_TRY(pairdiag_monopole(h, &dmin, &dmax, &pos));
            if (h->d_kmap) {                      // its kept index (the lowest state is always kept)
                int32_t m = -1;
                PD_CUDA(cudaMemcpy(&m, h->d_kmap + pos, sizeof m, cudaMemcpyDeviceToHost));
                if (m < 0) return fail(PD_ECUDA, "internal: the lowest state was dropped");
                pos = m;
            }
        }
        const size_t es = dtype == 0 ? 8 : 4;
        PD_CUDA(cudaMemsetAsync(q0, 0, es * (size_t)dim, h->st));
        const double one = 1.0;
        const float onef = 1.0f;
        PD_CUDA(cudaMemcpyAsync(static_cast<char *>(q0) + es * (size_t)pos, dtype == 0 ? (const void *)&one : (const void *)&onef,
                                es, cudaMemcpyHostToDevice, h->st));
        PD_CUDA(cudaStreamSynchronize(h->st));
        break;
    }
    case PD_START_MLP: {
        std::vector<double> w(h->omega);
        if (h->mlp) PD_TRY(mlp_predict(h->mlp, h->omega, h->n, h->e.data(), h->G.data(), w.data()));
        else if ((int)h->start_w.size() == h->omega) w = h->start_w;
        else return fail(PD_EINVAL, "PD_START_MLP needs pairdiag_set_mlp or pairdiag_set_start_weights");
        PD_TRY(product_start(h->B, w.data(), dtype, q0, h->st, factor_scratch(h)));
        break;
    }
    case PD_START_USER: {
        if ((int64_t)h->start.size() != dim) return fail(PD_EINVAL, "no start vector set (pairdiag_set_start)");
        PD_TRY(ensure_fp64_pair(h));
        PD_CUDA(cudaMemcpyAsync(h->d_v64, h->start.data(), sizeof(double) * dim, cudaMemcpyHostToDevice, h->st));
        PD_CUDA(convert_launch(dtype, q0, 0, h->d_v64, dim, h->st));
        break;
    }
    default:
        return fail(PD_EINVAL, "unknown start kind %d", h->opt.start);
    }
    return PD_OK;
}

// FP64 Rayleigh quotient and residual of Q_0 (of storage dtype): v64 <- Q_0,
// w64 <- H v64.  Returns lambda, relative residual ||Hv - lambda v|| / |lambda| / ||v||.
int rayleigh64(pairdiag *h, int dtype, double *lambda, double *rel)
{
    const int64_t dim = h->dim;
    PD_TRY(ensure_fp64_pair(h));
    PD_CUDA(convert_launch(0, h->d_v64, dtype, qvec(h, dtype, 0), dim, h->st));
    LanczosScalars *S = h->d_S;
    // w = H v with v^T w fused into the product; v^T v; lambda = v^T w / v^T v
    // and ||w - lambda v||^2 on the device; one synchronisation.  An FP32 v
    // (the mixed form) takes the float-float product: rows as accurate as FP64
    // sums, on the FP32 pipes
    if (dtype == 1 && h->hxgrid[2] > 0) PD_TRY(hx(h, 2, qvec(h, dtype, 0), h->d_w64, nullptr, &S->dots[0]));
    else PD_TRY(hx(h, 0, h->d_v64, h->d_w64, nullptr, &S->dots[0]));
    unsigned long long *tk = &h->d_tk->vec_done;
    PD_CUDA(multidot_launch(0, h->d_v64, dim, 1, h->d_v64, dim, h->d_part, &S->dots[1], h->st, nullptr, tk));
    PD_CUDA(quotient_launch(&S->dots[0], &S->dots[1], &S->dots[2], h->st));
    PD_CUDA(residual_launch(h->d_w64, h->d_v64, &S->dots[2], nullptr, dim, h->d_part, &S->dots[3], h->st, tk));
    double d[4];
    PD_CUDA(cudaMemcpyAsync(d, S->dots, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    const double lam = d[2], r2 = d[3];
    *lambda = lam;
    *rel = (r2 == 0.0) ? 0.0 : std::sqrt(r2 / d[1]) / std::fabs(lam);
    return PD_OK;
}

int ground_state_impl(pairdiag *h, double tol, double *e0, double *vec_dev, bool vec_is_host,
                      double *vec_host, pairdiag_info *info)
{
    if (!h || !e0) return fail(PD_EINVAL, "null argument");
    if (!(tol >= 0.0)) return fail(PD_EINVAL, "tol must be >= 0");
    const auto t0 = std::chrono::steady_clock::now();
    PD_CUDA(cudaSetDevice(h->device));
    const int64_t dim = h->dim;
    const int win = std::min<int64_t>(std::max(1, h->opt.window), std::min<int64_t>(dim, kMaxWindow));
    CycleStats cs;
    int status = PD_OK;
    int fp32_iters = 0;
    int refinements = 0;
    int final_dtype = 0;
    double energy = 0.0, rel = INFINITY;
    if (h->opt.precision == PD_PREC_MIXED) {
        PD_TRY(ensure_window(h, 1, win));
        PD_TRY(init_start(h, 1));
        const double tol32 = std::max(tol, h->opt.mixed_floor);
        PD_TRY(run_cycles(h, 1, tol32, h->opt.max_restarts, cs));
        fp32_iters = cs.iterations;
        double lam, r;
        PD_TRY(rayleigh64(h, 1, &lam, &r));
        ++refinements;
        energy = lam; rel = r;
        if (r <= tol || h->opt.mode == 1) {
            cs.converged = true;
            final_dtype = -1;                  // vector lives in d_v64
        } else {
            // continue in FP64 from the refined vector
            PD_TRY(ensure_window(h, 0, win));
            PD_CUDA(cudaMemcpyAsync(qvec(h, 0, 0), h->d_v64, sizeof(double) * dim, cudaMemcpyDeviceToDevice, h->st));
            CycleStats c64;
            const int left = std::max(0, h->opt.max_restarts - cs.restarts);
            PD_TRY(run_cycles(h, 0, tol, left, c64));
            cs.iterations += c64.iterations;
            cs.restarts += c64.restarts;
            cs.converged = c64.converged;
            cs.gap = c64.gap;
            energy = c64.energy;
            rel = c64.rel;
            final_dtype = 0;
        }
    } else {
        PD_TRY(ensure_window(h, 0, win));
        PD_TRY(init_start(h, 0));
        PD_TRY(run_cycles(h, 0, tol, h->opt.max_restarts, cs));
        energy = cs.energy;
        rel = cs.rel;
        final_dtype = 0;
        if (h->opt.mode == 1) {                // report the residual of the Ritz vector
            double lam, r;
            PD_TRY(rayleigh64(h, 0, &lam, &r));
            ++refinements;
            rel = r;
        }
    }
    if (!cs.converged) status = fail(PD_ENOCONV, "tolerance %.3g not reached after %d restarts (residual %.3g)",
                                     tol, cs.restarts, rel);
    // output vector
    const double *src = final_dtype == -1 ? h->d_v64 : static_cast<const double *>(qvec(h, 0, 0));
    if (final_dtype == -1) {                   // normalise the refined FP64 copy
        PD_CUDA(multidot_launch(0, h->d_v64, dim, 1, h->d_v64, dim, h->d_part, &h->d_S->dots[0], h->st, nullptr,
                                &h->d_tk->vec_done));
        PD_CUDA(scale_launch(0, h->d_v64, h->d_v64, dim, &h->d_S->dots[0], 1, h->st));
    }
    if (vec_dev) PD_CUDA(cudaMemcpyAsync(vec_dev, src, sizeof(double) * dim, cudaMemcpyDeviceToDevice, h->st));
    if (vec_is_host && vec_host)
        PD_CUDA(cudaMemcpyAsync(vec_host, src, sizeof(double) * dim, cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    *e0 = energy;
    if (info) {
        info->dim = dim;
        info->nnz_offdiag = h->nnz;
        info->iterations = cs.iterations;
        info->hx_products = cs.iterations + refinements;
        info->iterations_fp32 = fp32_iters;
        info->restarts = cs.restarts;
        info->converged = cs.converged ? 1 : 0;
        info->rel_residual = rel;
        info->gap_estimate = cs.gap;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}

}  // namespace

extern "C" {

void pairdiag_default_options(pairdiag_options *opt)
{
    if (!opt) return;
    opt->window = 20;
    opt->max_restarts = 500;
    opt->precision = PD_PREC_FP64;
    opt->start = PD_START_RANDOM;
    opt->seed = 1;
    opt->mode = 0;
    opt->low_bits = 0;
    opt->mixed_floor = 5e-6;
    opt->hx_variant = 0;
}

const char *pairdiag_strerror(int code)
{
    switch (code) {
    case PD_OK: return "success";
    case PD_EINVAL: return "invalid argument";
    case PD_ENOMEM: return "out of device memory";
    case PD_ENOCONV: return "Lanczos did not converge";
    case PD_ETIMEOUT: return "device wait timed out";
    case PD_ECUDA: return "CUDA error";
    case PD_ENOTSUP: return "not supported";
    default: return "unknown status";
    }
}

const char *pairdiag_last_error(void) { return g_last_error.c_str(); }

int pairdiag_create(int omega, int n_pairs, const double *e, const double *G,
                    const pairdiag_options *opt, pairdiag_t **out)
{
    if (!out) return fail(PD_EINVAL, "out is null");
    *out = nullptr;
    if (omega < 1 || omega > kMaxOmega) return fail(PD_EINVAL, "omega=%d outside 1..%d", omega, kMaxOmega);
    if (n_pairs < 0 || n_pairs > omega) return fail(PD_EINVAL, "n_pairs=%d outside 0..omega", n_pairs);
    if (!e || !G) return fail(PD_EINVAL, "e or G is null");
    for (int i = 0; i < omega; ++i)
        if (!std::isfinite(e[i])) return fail(PD_EINVAL, "e[%d] is not finite", i);
    for (int i = 0; i < omega; ++i)
        for (int j = 0; j < omega; ++j) {
            if (!std::isfinite(G[i * omega + j])) return fail(PD_EINVAL, "G[%d][%d] is not finite", i, j);
            if (G[i * omega + j] != G[j * omega + i]) return fail(PD_EINVAL, "G is not symmetric at (%d,%d)", i, j);
        }
    pairdiag_options o;
    pairdiag_default_options(&o);
    if (opt) o = *opt;
    if (o.window < 1 || o.window > kMaxWindow) return fail(PD_EINVAL, "window=%d outside 1..%d", o.window, kMaxWindow);
    if (o.precision != PD_PREC_FP64 && o.precision != PD_PREC_MIXED) return fail(PD_EINVAL, "bad precision");
    if (o.mode != 0 && o.mode != 1) return fail(PD_EINVAL, "bad mode");
    if (o.low_bits < 0 || o.low_bits > kMaxLow) return fail(PD_EINVAL, "low_bits outside 0..%d", kMaxLow);
    if (o.max_restarts < 0) return fail(PD_EINVAL, "max_restarts < 0");
    if (o.hx_variant < 0 || o.hx_variant > 5) return fail(PD_EINVAL, "hx_variant outside 0..5");
    if (o.start < PD_START_RANDOM || o.start > PD_START_MLP) return fail(PD_EINVAL, "bad start kind");

    if (o.low_bits == 0 && o.hx_variant == 0) {   // an autotuned schedule, if one was recorded
        int lb = 0, hv = 0;
        if (tuned_schedule(omega, n_pairs, o.precision, &lb, &hv)) { o.low_bits = lb; o.hx_variant = hv; }
    }
    if (o.hx_variant == 0) {
        // untuned: direct gathers; far from half filling (fewer than 3 in 10 orbits
        // occupied, or empty) deep gather groups and 13 low orbits, the fastest
        // schedules measured at Omega = 24..38
        const int minority = std::min(n_pairs, omega - n_pairs);
        const bool low_filling = 10 * minority < 3 * omega;
        o.hx_variant = low_filling ? 4 : 3;
        if (o.low_bits == 0 && low_filling) o.low_bits = 13;
    }
    pairdiag *h = new pairdiag();
    h->omega = omega; h->n = n_pairs; h->opt = o;
    h->e.assign(e, e + omega);
    h->G.assign(G, G + (size_t)omega * omega);
    h->d.resize(omega);
    for (int p = 0; p < omega; ++p) h->d[p] = 2.0 * e[p] + G[p * omega + p];
    h->dim = (int64_t)host_binom(omega, n_pairs);
    h->nnz = h->dim * (int64_t)n_pairs * (int64_t)(omega - n_pairs);
    h->full_dim = h->dim;
    h->full_nnz = h->nnz;
    int st = PD_OK;
    do {
        if (cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); st = fail(PD_ECUDA, "no CUDA device"); break; }
        if ((st = build_tables(h)) != PD_OK) break;
        std::vector<float> G32(h->G.begin(), h->G.end()), d32(h->d.begin(), h->d.end());
        auto split = [](const std::vector<double> &v) {
            std::vector<float2> r(v.size());
            for (size_t i = 0; i < v.size(); ++i) {
                const float hi = (float)v[i];
                r[i] = make_float2(hi, (float)(v[i] - (double)hi));
            }
            return r;
        };
        if ((st = upload(&h->d_G64, h->G)) != PD_OK) break;
        if ((st = upload(&h->d_d64, h->d)) != PD_OK) break;
        if ((st = upload(&h->d_G32, G32)) != PD_OK) break;
        if ((st = upload(&h->d_d32, d32)) != PD_OK) break;
        if ((st = upload(&h->d_Gff, split(h->G))) != PD_OK) break;
        if ((st = upload(&h->d_dff, split(h->d))) != PD_OK) break;
        if ((st = dalloc(&h->d_tk, 1)) != PD_OK) break;
        if (cudaMemset(h->d_tk, 0, sizeof(Tickets)) != cudaSuccess) { st = fail(PD_ECUDA, "memset"); break; }
        if ((st = dalloc(&h->d_blkdot, (size_t)h->B.nblocks)) != PD_OK) break;
        h->ldq = (h->dim + 3) / 4 * 4;
        h->hxgrid[0] = hx_grid(h->B, 0);
        h->hxgrid[1] = hx_grid(h->B, 1);
        h->hxgrid[2] = hx_grid(h->B, 2);
        h->rgrid = (int)std::min<int64_t>(h->B.nblocks, vec_grid());
        h->part_count = (size_t)std::max(vec_grid(), h->rgrid) * kMaxWindow;
        if ((st = dalloc(&h->d_part, h->part_count)) != PD_OK) break;
        if ((st = dalloc(&h->d_S, 1)) != PD_OK) break;
        if ((st = dalloc(&h->d_small, 8)) != PD_OK) break;
        if (cudaMemset(h->d_S, 0, sizeof(LanczosScalars)) != cudaSuccess) { st = fail(PD_ECUDA, "memset"); break; }
    } while (0);
    if (st != PD_OK) {
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return PD_OK;
}

void pairdiag_destroy(pairdiag_t *h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    free_all(h);
    delete h;
}

int64_t pairdiag_kernel_launches(void) { return (int64_t)g_kernel_launches.load(); }

int pairdiag_set_profiling(pairdiag_t *h, int on)
{
    if (!h) return fail(PD_EINVAL, "null handle");
    h->profiling = on != 0;
    return PD_OK;
}

int pairdiag_set_step_fusion(pairdiag_t *h, int on)
{
    if (!h) return fail(PD_EINVAL, "null handle");
    h->step_fusion = on != 0;
    return PD_OK;
}

int pairdiag_get_profile(pairdiag_t *h, int precision, int64_t *hx_launches, double *hx_ms)
{
    if (!h || !hx_launches || !hx_ms) return fail(PD_EINVAL, "null argument");
    PD_CUDA(cudaStreamSynchronize(h->st));
    double total = 0.0;
    int64_t count = 0;
    size_t kept = 0;                              // records of other precisions stay, in order
    for (size_t i = 0; i < h->hx_events_used; ++i) {
        const int code = h->hx_event_prec[i];
        if (precision >= 0 ? code != precision : code >= 2) {
            std::swap(h->hx_events[kept], h->hx_events[i]);
            std::swap(h->hx_event_prec[kept], h->hx_event_prec[i]);
            ++kept;
            continue;
        }
        float ms = 0.0f;
        PD_CUDA(cudaEventElapsedTime(&ms, h->hx_events[i].first, h->hx_events[i].second));
        total += ms;
        ++count;
    }
    *hx_launches = count;
    *hx_ms = total;
    h->hx_events_used = kept;
    return PD_OK;
}

int pairdiag_set_stream(pairdiag_t *h, void *stream)
{
    if (!h) return fail(PD_EINVAL, "null handle");
    h->st = static_cast<cudaStream_t>(stream);
    return PD_OK;
}

int64_t pairdiag_dim(const pairdiag_t *h) { return h ? h->dim : -1; }
int64_t pairdiag_nnz(const pairdiag_t *h) { return h ? h->nnz : -1; }
int pairdiag_omega(const pairdiag_t *h) { return h ? h->omega : -1; }

int pairdiag_basis_dev(const pairdiag_t *h, int64_t first, int64_t count, uint64_t *out_dev)
{
    if (!h || (!out_dev && count > 0)) return fail(PD_EINVAL, "null argument");
    if (first < 0 || count < 0 || first + count > h->full_dim)
        return fail(PD_EINVAL, "range outside [0, C(omega, n_pairs))");
    PD_CUDA(basis_launch(h->omega, h->n, h->d_binom, first, count, out_dev, h->st));
    return PD_OK;
}

int pairdiag_basis(const pairdiag_t *h, uint64_t *out)
{
    if (!h || !out) return fail(PD_EINVAL, "null argument");
    uint64_t *d = nullptr;
    PD_TRY(dalloc(&d, (size_t)h->full_dim));
    int st = pairdiag_basis_dev(h, 0, h->full_dim, d);
    if (st == PD_OK) {
        cudaError_t e1 = cudaMemcpyAsync(out, d, sizeof(uint64_t) * h->full_dim, cudaMemcpyDeviceToHost, h->st);
        cudaError_t e2 = cudaStreamSynchronize(h->st);
        if (e1 != cudaSuccess || e2 != cudaSuccess) st = fail(PD_ECUDA, "basis copy failed");
    }
    cudaStreamSynchronize(h->st);
    pool_free(d);
    return st;
}

int pairdiag_rank_dev(const pairdiag_t *h, const uint64_t *states_dev, int64_t count, uint64_t *ranks_dev)
{
    if (!h || ((!states_dev || !ranks_dev) && count > 0) || count < 0) return fail(PD_EINVAL, "bad argument");
    PD_CUDA(rank_launch(h->omega, h->n, h->d_binom, states_dev, count, ranks_dev, h->st));
    return PD_OK;
}

int pairdiag_hx_dev(pairdiag_t *h, int precision, const void *x_dev, void *y_dev)
{
    if (!h || !x_dev || !y_dev) return fail(PD_EINVAL, "null argument");
    if (precision != PD_PREC_FP64 && precision != PD_PREC_MIXED && precision != PD_HX_FLOATFLOAT)
        return fail(PD_EINVAL, "bad precision");
    if (x_dev == y_dev) return fail(PD_EINVAL, "x and y must not overlap");
    if (precision == PD_HX_FLOATFLOAT && h->hxgrid[2] < 1)
        return fail(PD_ENOTSUP, "no float-float product for this handle (truncated space or shared memory)");
    return hx(h, precision, x_dev, y_dev);
}

int pairdiag_hx(pairdiag_t *h, const double *x, double *y)
{
    if (!h || !x || !y) return fail(PD_EINVAL, "null argument");
    PD_TRY(ensure_fp64_pair(h));
    PD_CUDA(cudaMemcpyAsync(h->d_v64, x, sizeof(double) * h->dim, cudaMemcpyHostToDevice, h->st));
    PD_TRY(hx(h, 0, h->d_v64, h->d_w64));
    PD_CUDA(cudaMemcpyAsync(y, h->d_w64, sizeof(double) * h->dim, cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    return PD_OK;
}

int pairdiag_monopole(pairdiag_t *h, double *dmin, double *dmax, int64_t *pos_min)
{
    if (!h || !dmin || !dmax || !pos_min) return fail(PD_EINVAL, "null argument");
    PD_CUDA(monopole_launch(h->B, h->d_d64, h->d_part, h->rgrid, h->d_small, h->st));
    double out[3];
    PD_CUDA(cudaMemcpyAsync(out, h->d_small, sizeof out, cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    *dmin = out[0];
    *dmax = out[1];
    int64_t pos;
    memcpy(&pos, &out[2], sizeof pos);
    *pos_min = pos;
    return PD_OK;
}

int pairdiag_set_mlp(pairdiag_t *h, pairdiag_mlp_t *m)
{
    if (!h) return fail(PD_EINVAL, "null handle");
    h->mlp = m;
    return PD_OK;
}

int pairdiag_set_start_weights(pairdiag_t *h, const double *w)
{
    if (!h || !w) return fail(PD_EINVAL, "null argument");
    h->start_w.assign(w, w + h->omega);
    return PD_OK;
}

int pairdiag_product_fit(pairdiag_t *h, const double *v_dev, double *w)
{
    if (!h || !v_dev || !w) return fail(PD_EINVAL, "null argument");
    if (h->d_kmap) return fail(PD_ENOTSUP, "product fit of a truncated space");
    return product_fit(h->B, v_dev, w, h->st);
}

int pairdiag_product_start_dev(pairdiag_t *h, const double *w, double *v_dev)
{
    if (!h || !w || !v_dev) return fail(PD_EINVAL, "null argument");
    PD_TRY(product_start(h->B, w, 0, v_dev, h->st, factor_scratch(h)));
    PD_CUDA(cudaStreamSynchronize(h->st));
    return PD_OK;
}

int pairdiag_set_start(pairdiag_t *h, const double *v)
{
    if (!h || !v) return fail(PD_EINVAL, "null argument");
    h->start.assign(v, v + h->dim);
    return PD_OK;
}

int pairdiag_ground_state(pairdiag_t *h, double tol, double *e0, double *vec, pairdiag_info *info)
{
    return ground_state_impl(h, tol, e0, nullptr, true, vec, info);
}

int pairdiag_ground_state_dev(pairdiag_t *h, double tol, double *e0, double *vec_dev, pairdiag_info *info)
{
    return ground_state_impl(h, tol, e0, vec_dev, false, nullptr, info);
}

int pairdiag_occupations_dev(pairdiag_t *h, const double *v_dev, double *occ)
{
    if (!h || !v_dev || !occ) return fail(PD_EINVAL, "null argument");
    PD_CUDA(occupations_launch(h->B, v_dev, h->d_part, h->rgrid, h->d_S->s, h->st));
    PD_CUDA(cudaMemcpyAsync(occ, h->d_S->s, sizeof(double) * h->omega, cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    return PD_OK;
}

int pairdiag_lowest_states_dev(pairdiag_t *h, int k, double tol, double *energies, double *vecs_dev,
                               pairdiag_info *info)
{
    if (!h || !energies) return fail(PD_EINVAL, "null argument");
    if (k < 1 || k > kMaxWindow || (int64_t)k > h->dim)
        return fail(PD_EINVAL, "k=%d outside 1..min(%d, dim)", k, kMaxWindow);
    if (!(tol >= 0.0)) return fail(PD_EINVAL, "tol must be >= 0");
    PD_CUDA(cudaSetDevice(h->device));
    const int64_t dim = h->dim, ld = h->ldq;
    const bool mixed = h->opt.precision == PD_PREC_MIXED;
    if (h->lock_cap < k || (mixed && !h->d_L32)) {
        PD_CUDA(cudaStreamSynchronize(h->st));
        pool_free(h->d_L64);
        pool_free(h->d_L32);
        h->d_L64 = nullptr;
        h->d_L32 = nullptr;
        h->lock_cap = 0;
        PD_TRY(dalloc(&h->d_L64, (size_t)k * (size_t)ld));
        if (mixed) PD_TRY(dalloc(&h->d_L32, (size_t)k * (size_t)ld));
        h->lock_cap = k;
    }
    if (!h->d_lockc) PD_TRY(dalloc(&h->d_lockc, (size_t)kMaxWindow));
    int status = PD_OK;
    h->n_locked = 0;
    // state 0 starts as the handle's options say; every later state from its own
    // random vector: a start reused after projection has no component left in
    // the rest of a degenerate eigenspace, so Lanczos would skip its other copies
    const int start0 = h->opt.start;
    const uint64_t seed0 = h->opt.seed;
    auto restore = [&]() {
        h->n_locked = 0;
        h->opt.start = start0;
        h->opt.seed = seed0;
    };
    for (int j = 0; j < k; ++j) {
        if (j > 0) {
            h->opt.start = PD_START_RANDOM;
            h->opt.seed = seed0 + (uint64_t)j;
        }
        double ej = 0.0;
        double *slot = h->d_L64 + (size_t)j * (size_t)ld;
        const int st = ground_state_impl(h, tol, &ej, slot, false, nullptr, info ? &info[j] : nullptr);
        if (st != PD_OK && st != PD_ENOCONV) {
            restore();
            return st;
        }
        if (st == PD_ENOCONV) status = PD_ENOCONV;
        energies[j] = ej;
        if (h->d_L32) {
            const cudaError_t ce = convert_launch(1, h->d_L32 + (size_t)j * (size_t)ld, 0, slot, dim, h->st);
            if (ce != cudaSuccess) {
                restore();
                return fail(PD_ECUDA, "convert: %s", cudaGetErrorString(ce));
            }
        }
        h->n_locked = j + 1;
    }
    restore();                                    // later ground-state calls see the whole space
    if (vecs_dev)
        PD_CUDA(cudaMemcpy2DAsync(vecs_dev, sizeof(double) * (size_t)dim, h->d_L64, sizeof(double) * (size_t)ld,
                                  sizeof(double) * (size_t)dim, (size_t)k, cudaMemcpyDeviceToDevice, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    if (status == PD_ENOCONV) return fail(PD_ENOCONV, "a state missed tol %.3g", tol);
    return PD_OK;
}

// ---- truncated model space (Sec. 3.5) ---------------------------------------------
namespace {

constexpr int kHistBuckets = 8192;   // buckets per histogram pass
constexpr int64_t kMaxBins = (int64_t)1 << 40;

// back to the full space: drop the map and every vector sized by the old space
void drop_space(pairdiag *h)
{
    cudaStreamSynchronize(h->st);
    void **vecs[] = {&h->d_Q[0], &h->d_Q[1], &h->d_p[0], &h->d_p[1], (void **)&h->d_v64, (void **)&h->d_w64,
                     (void **)&h->d_L64, (void **)&h->d_L32, (void **)&h->d_kmap, (void **)&h->d_kblk_h,
                     (void **)&h->d_kblk_base};
    for (void **v : vecs) {
        pool_free(*v);
        *v = nullptr;
    }
    h->Qwin[0] = h->Qwin[1] = 0;
    h->lock_cap = 0;
    h->n_locked = 0;
    h->start.clear();
    h->B.kept_map = nullptr;
    h->B.kept_blk_h = h->B.kept_blk_base = nullptr;
    h->B.kept_nblocks = 0;
    h->dim = h->full_dim;
    h->nnz = h->full_nnz;
    h->ldq = (h->dim + 3) / 4 * 4;
    h->hxgrid[0] = hx_grid(h->B, 0);
    h->hxgrid[1] = hx_grid(h->B, 1);
    h->hxgrid[2] = hx_grid(h->B, 2);
}

// The kept states of Sec. 3.5 and the map full index -> kept index.  Returns
// the kept count in *kept (== full_dim when nothing is dropped, no map made).
int build_truncation(pairdiag *h, int64_t limit, int64_t bins, int64_t *kept)
{
    const int64_t full = h->full_dim;
    *kept = full;
    if (limit >= full) return PD_OK;                 // no truncation
    double lo, hi;
    int64_t pos;
    PD_TRY(pairdiag_monopole(h, &lo, &hi, &pos));
    if (!(hi > lo)) return PD_OK;                     // every diagonal element equal
    const Blocks &B = h->B;
    const int grid = h->rgrid;
    cudaStream_t st = h->st;
    std::vector<void *> tmp;
    auto cleanup = [&]() {
        cudaStreamSynchronize(st);
        for (void *p : tmp) pool_free(p);
    };
    auto talloc = [&](void **p, size_t bytes) -> int {
        const cudaError_t e = pool_alloc(p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PD_ENOMEM, "truncation: %zu bytes: %s", bytes, cudaGetErrorString(e));
        }
        tmp.push_back(*p);
        return PD_OK;
    };
    int rc = [&]() -> int {
        // the cutoff bin: the lowest bin at which the running count reaches the
        // limit, found by histograms over ever narrower bin ranges
        unsigned long long *hist = nullptr;
        PD_TRY(talloc((void **)&hist, sizeof(unsigned long long) * kHistBuckets));
        std::vector<unsigned long long> hh(kHistBuckets);
        int64_t lo_bin = 0, span = bins;
        unsigned long long below = 0;                 // states in bins below lo_bin
        const unsigned long long need = (unsigned long long)limit;
        int64_t cut = -1;
        for (int level = 0; level < 8 && cut < 0; ++level) {
            int shift = 0;
            while (((span + ((int64_t)1 << shift) - 1) >> shift) > kHistBuckets) ++shift;
            const int nb = (int)((span + ((int64_t)1 << shift) - 1) >> shift);
            PD_CUDA(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * nb, st));
            PD_CUDA(trunc_hist_launch(B, h->d_d64, lo, hi, bins, lo_bin, shift, nb, hist, grid, st));
            PD_CUDA(cudaMemcpyAsync(hh.data(), hist, sizeof(unsigned long long) * nb, cudaMemcpyDeviceToHost, st));
            PD_CUDA(cudaStreamSynchronize(st));
            int j = 0;
            unsigned long long run = below;
            while (j < nb && run + hh[j] < need) run += hh[j++];
            if (j == nb) return fail(PD_ECUDA, "internal: truncation histogram holds %llu of %lld states",
                                     run, (long long)limit);
            below = run;
            lo_bin += (int64_t)j << shift;
            if (shift == 0) cut = lo_bin;
            else span = std::min<int64_t>((int64_t)1 << shift, bins - lo_bin);
        }
        if (cut < 0) return fail(PD_ECUDA, "internal: truncation cutoff not found");
        // kept states per block, their first kept index, and the map
        int *blk_kept = nullptr;
        PD_TRY(talloc((void **)&blk_kept, sizeof(int) * (size_t)B.nblocks));
        PD_CUDA(trunc_count_launch(B, h->d_d64, lo, hi, bins, cut, blk_kept, grid, st));
        std::vector<int> cnt((size_t)B.nblocks);
        PD_CUDA(cudaMemcpyAsync(cnt.data(), blk_kept, sizeof(int) * cnt.size(), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaStreamSynchronize(st));
        std::vector<int64_t> first(cnt.size());
        int64_t total = 0;
        for (size_t b = 0; b < cnt.size(); ++b) {
            first[b] = total;
            total += cnt[b];
        }
        if (total < limit || total > full) return fail(PD_ECUDA, "internal: %lld states kept", (long long)total);
        *kept = total;
        if (total == full) return PD_OK;              // the cutoff bin is the last one
        if (total > (int64_t)INT32_MAX) return fail(PD_ENOTSUP, "more than 2^31 - 1 kept states");
        int64_t *d_first = nullptr;
        PD_TRY(talloc((void **)&d_first, sizeof(int64_t) * first.size()));
        PD_CUDA(cudaMemcpyAsync(d_first, first.data(), sizeof(int64_t) * first.size(), cudaMemcpyHostToDevice, st));
        PD_TRY(dalloc(&h->d_kmap, (size_t)full));
        PD_CUDA(trunc_map_launch(B, h->d_d64, lo, hi, bins, cut, d_first, h->d_kmap, grid, st));
        // the blocks that hold kept states, for the truncated H*x to walk
        std::vector<uint64_t> bh(cnt.size()), bb(cnt.size());
        PD_CUDA(cudaMemcpyAsync(bh.data(), B.blk_h, sizeof(uint64_t) * bh.size(), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaMemcpyAsync(bb.data(), B.blk_base, sizeof(uint64_t) * bb.size(), cudaMemcpyDeviceToHost, st));
        PD_CUDA(cudaStreamSynchronize(st));
        std::vector<uint64_t> kh, kb;
        for (size_t b = 0; b < cnt.size(); ++b)
            if (cnt[b] > 0) {
                kh.push_back(bh[b]);
                kb.push_back(bb[b]);
            }
        PD_TRY(upload(&h->d_kblk_h, kh));
        PD_TRY(upload(&h->d_kblk_base, kb));
        h->B.kept_nblocks = (int64_t)kh.size();
        return PD_OK;
    }();
    cleanup();
    return rc;
}

}  // namespace

int pairdiag_truncate(pairdiag_t *h, int64_t dimension_limit, int64_t bins, int64_t *kept_dim)
{
    if (!h || !kept_dim) return fail(PD_EINVAL, "null argument");
    if (dimension_limit < 0) return fail(PD_EINVAL, "dimension_limit < 0");
    if (bins == 0) bins = 100000000;
    if (bins < 1 || bins > kMaxBins) return fail(PD_EINVAL, "bins outside 1..2^40");
    PD_CUDA(cudaSetDevice(h->device));
    drop_space(h);
    *kept_dim = h->dim;
    if (dimension_limit == 0) return PD_OK;
    int64_t kept = 0;
    int rc = build_truncation(h, dimension_limit, bins, &kept);
    if (rc == PD_OK && h->d_kmap) {
        h->dim = kept;
        h->ldq = (kept + 3) / 4 * 4;
        h->B.kept_map = h->d_kmap;
        h->B.kept_blk_h = h->d_kblk_h;
        h->B.kept_blk_base = h->d_kblk_base;
        h->hxgrid[0] = hx_grid(h->B, 0);
        h->hxgrid[1] = hx_grid(h->B, 1);
        h->hxgrid[2] = hx_grid(h->B, 2);
        // off-diagonal nonzeros of the truncated matrix: H x with every G_ij = 1
        // and d = 0 on x = 1 counts each row's kept targets (exact in FP64)
        rc = [&]() -> int {
            std::vector<double> ones((size_t)h->omega * h->omega, 1.0), zeros(h->omega, 0.0);
            double *g1 = nullptr, *d0 = nullptr;
            PD_TRY(upload(&g1, ones));
            const int r0 = upload(&d0, zeros);
            if (r0 != PD_OK) { pool_free(g1); return r0; }
            int r = ensure_fp64_pair(h);
            if (r == PD_OK) r = product_start(h->B, zeros.data(), 0, h->d_v64, h->st);   // kept entries = 1
            if (r == PD_OK && cudaStreamSynchronize(h->st) != cudaSuccess) r = fail(PD_ECUDA, "product start");
            if (r == PD_OK) {
                const HxProblem P1{g1, d0, nullptr, nullptr};
                cudaError_t ce = hx_launch(h->B, P1, 0, h->d_v64, h->d_w64, h->d_tk, h->hxgrid[0], h->st);
                if (ce == cudaSuccess)
                    ce = multidot_launch(0, h->d_w64, kept, 1, h->d_v64, kept, h->d_part, &h->d_S->dots[0], h->st,
                                         nullptr, &h->d_tk->vec_done);
                double c = 0.0;
                if (ce == cudaSuccess) ce = cudaMemcpyAsync(&c, &h->d_S->dots[0], sizeof c, cudaMemcpyDeviceToHost, h->st);
                if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->st);
                if (ce != cudaSuccess) r = fail(PD_ECUDA, "truncation nonzero count: %s", cudaGetErrorString(ce));
                else h->nnz = (int64_t)std::llround(c);
            }
            cudaStreamSynchronize(h->st);
            pool_free(g1);
            pool_free(d0);
            return r;
        }();
    }
    if (rc != PD_OK) {
        drop_space(h);
        return rc;
    }
    *kept_dim = h->dim;
    return PD_OK;
}

int pairdiag_kept_map_dev(const pairdiag_t *h, int32_t *map_dev)
{
    if (!h || !map_dev) return fail(PD_EINVAL, "null argument");
    if (!h->d_kmap) return fail(PD_EINVAL, "the handle holds the full space (no truncation active)");
    PD_CUDA(cudaMemcpyAsync(map_dev, h->d_kmap, sizeof(int32_t) * (size_t)h->full_dim, cudaMemcpyDeviceToDevice,
                            h->st));
    return PD_OK;
}

int64_t pairdiag_full_dim(const pairdiag_t *h) { return h ? h->full_dim : -1; }

int pairdiag_multidot(pairdiag_t *h, int dtype, const void *Q_dev, int64_t ld, int m, const void *p_dev,
                      int64_t n, double *out)
{
    if (!h || !Q_dev || !p_dev || !out) return fail(PD_EINVAL, "null argument");
    if (m < 1 || m > kMaxWindow || n < 0 || ld < n || (dtype != 0 && dtype != 1))
        return fail(PD_EINVAL, "bad sizes (need 1 <= m <= %d, 0 <= n <= ld, dtype 0 or 1)", kMaxWindow);
    PD_CUDA(multidot_launch(dtype, Q_dev, ld, m, p_dev, n, h->d_part, h->d_S->c1, h->st, nullptr,
                            &h->d_tk->vec_done));
    PD_CUDA(cudaMemcpyAsync(out, h->d_S->c1, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    return PD_OK;
}

int pairdiag_tridiag_lowest(pairdiag_t *h, int m, const double *alpha, const double *beta, double *theta,
                            double *s)
{
    if (!h || !alpha || !theta || !s || (m > 1 && !beta)) return fail(PD_EINVAL, "null argument");
    if (m < 1 || m > kMaxWindow) return fail(PD_EINVAL, "m outside 1..%d", kMaxWindow);
    LanczosScalars *S = h->d_S;
    PD_CUDA(cudaMemcpyAsync(S->alpha, alpha, sizeof(double) * m, cudaMemcpyHostToDevice, h->st));
    if (m > 1) PD_CUDA(cudaMemcpyAsync(S->beta, beta, sizeof(double) * (m - 1), cudaMemcpyHostToDevice, h->st));
    PD_CUDA(tridiag_launch(S, m, h->st));
    PD_CUDA(cudaMemcpyAsync(theta, S->theta, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaMemcpyAsync(s, S->s, sizeof(double) * m, cudaMemcpyDeviceToHost, h->st));
    PD_CUDA(cudaStreamSynchronize(h->st));
    return PD_OK;
}

// ---- autotuner ------------------------------------------------------------------
int pairdiag_autotune(int omega, int n_pairs, const double *e, const double *G, int precision, int reps,
                      pairdiag_tune_entry *best, pairdiag_tune_entry *all, int *n_all)
{
    if (!e || !G || !best || reps < 1) return fail(PD_EINVAL, "bad argument");
    if (precision != PD_PREC_FP64 && precision != PD_PREC_MIXED) return fail(PD_EINVAL, "bad precision");
    if (omega < 1 || omega > kMaxOmega || n_pairs < 0 || n_pairs > omega) return fail(PD_EINVAL, "bad size");
    const int lmax = std::min(omega, kMaxLow), lmin = std::max(1, std::min(omega, 8));
    std::vector<pairdiag_tune_entry> res;
    const size_t es = precision == PD_PREC_FP64 ? 8 : 4;
    const int64_t dim = (int64_t)host_binom(omega, n_pairs);
    void *x = nullptr, *y = nullptr;
    PD_CUDA(cudaMalloc(&x, es * (size_t)dim));
    cudaError_t ce = cudaMalloc(&y, es * (size_t)dim);
    if (ce != cudaSuccess) { cudaFree(x); PD_CUDA(ce); }
    int rc = PD_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int L = lmin; L <= lmax && rc == PD_OK; ++L) {
        for (int variant = 1; variant <= 5 && rc == PD_OK; ++variant) {
            pairdiag_options o;
            pairdiag_default_options(&o);
            o.low_bits = L;
            o.hx_variant = variant;
            o.precision = precision;
            pairdiag_t *h = nullptr;
            if ((rc = pairdiag_create(omega, n_pairs, e, G, &o, &h)) != PD_OK) break;
            if (variant > 1 && hx_variant(h->B, precision == PD_PREC_FP64 ? 0 : 1) != variant) {
                pairdiag_destroy(h);             // the variant does not fit: same as variant 1
                continue;
            }
            rc = [&]() -> int {
                PD_CUDA(random_start_launch(precision == PD_PREC_FP64 ? 0 : 1, x, dim, 7, h->st));
                for (int w = 0; w < 2; ++w) PD_TRY(hx(h, precision == PD_PREC_FP64 ? 0 : 1, x, y));
                std::vector<float> t(reps);
                for (int r = 0; r < reps; ++r) {
                    PD_CUDA(cudaEventRecord(e0, h->st));
                    PD_TRY(hx(h, precision == PD_PREC_FP64 ? 0 : 1, x, y));
                    PD_CUDA(cudaEventRecord(e1, h->st));
                    PD_CUDA(cudaEventSynchronize(e1));
                    PD_CUDA(cudaEventElapsedTime(&t[r], e0, e1));
                }
                std::sort(t.begin(), t.end());
                res.push_back(pairdiag_tune_entry{L, variant, (double)t[reps / 2]});
                return PD_OK;
            }();
            pairdiag_destroy(h);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(y);
    if (rc != PD_OK) return rc;
    if (res.empty()) return fail(PD_ECUDA, "autotune: no candidate ran");
    const auto it = std::min_element(res.begin(), res.end(),
                                     [](const pairdiag_tune_entry &a, const pairdiag_tune_entry &b) { return a.ms < b.ms; });
    *best = *it;
    if (all && n_all) {
        const int cap = *n_all;
        int k = 0;
        for (const auto &r : res)
            if (k < cap) all[k++] = r;
        *n_all = k;
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune[TuneKey{omega, n_pairs, precision}] = {best->low_bits, best->hx_variant};
    }
    return PD_OK;
}

int pairdiag_tune_set(int omega, int n_pairs, int precision, int low_bits, int hx_variant_)
{
    if (low_bits < 0 || low_bits > kMaxLow || hx_variant_ < 0 || hx_variant_ > 5) return fail(PD_EINVAL, "bad schedule");
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    if (low_bits == 0) g_tune.erase(TuneKey{omega, n_pairs, precision});
    else g_tune[TuneKey{omega, n_pairs, precision}] = {low_bits, hx_variant_};
    return PD_OK;
}

int pairdiag_tune_get(int omega, int n_pairs, int precision, int *low_bits, int *hx_variant_)
{
    if (!low_bits || !hx_variant_) return fail(PD_EINVAL, "null argument");
    if (!tuned_schedule(omega, n_pairs, precision, low_bits, hx_variant_)) { *low_bits = 0; *hx_variant_ = 0; }
    return PD_OK;
}

}  // extern "C"

// ---- FMA throughput microbenchmark ---------------------------------------------
namespace {

constexpr int kFmaChains = 8;        // independent chains per thread
constexpr int kFmaIters = 4096;      // FMAs per chain

// x <- x a + b on kFmaChains independent chains; a = 1 - 2^-20 and b small keep
// every value bounded.  The sum is stored only when it equals an impossible
// value, so nothing is written and nothing can be optimised away.
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(T a, T b, T *sink)
{
    T x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
    for (int i = 0; i < kFmaIters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (s == T(-1.25e30)) *sink = s;
}

template <typename T>
int fma_peak_t(int reps, cudaStream_t st, double *tflops)
{
    int dev = 0, sms = 0, per_sm = 0;
    PD_CUDA(cudaGetDevice(&dev));
    PD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<T>, 256, 0));
    const int grid = sms * std::max(1, per_sm) * 4;
    T *sink = nullptr;
    PD_CUDA(cudaMalloc(&sink, sizeof(T)));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> ms(reps);
    int rc = PD_OK;
    const T a = T(1) - T(1) / T(1 << 20), b = T(1e-6);
    fma_peak_kernel<T><<<grid, 256, 0, st>>>(a, b, sink);            // warm-up
    count_launches(1);
    for (int r = 0; r < reps && rc == PD_OK; ++r) {
        cudaEventRecord(e0, st);
        fma_peak_kernel<T><<<grid, 256, 0, st>>>(a, b, sink);
        count_launches(1);
        cudaEventRecord(e1, st);
        const cudaError_t ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) rc = fail(PD_ECUDA, "fma_peak: %s", cudaGetErrorString(ce));
        else cudaEventElapsedTime(&ms[r], e0, e1);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc != PD_OK) return rc;
    std::sort(ms.begin(), ms.end());
    const double fmas = (double)grid * 256.0 * kFmaChains * kFmaIters;
    *tflops = 2.0 * fmas / (ms[reps / 2] * 1e-3) / 1e12;
    return PD_OK;
}

}  // namespace

extern "C" {

int pairdiag_fma_peak(int precision, int reps, void *stream, double *tflops)
{
    if (!tflops || reps < 1) return fail(PD_EINVAL, "bad argument");
    if (precision != PD_PREC_FP64 && precision != PD_PREC_MIXED) return fail(PD_EINVAL, "bad precision");
    const cudaStream_t st = static_cast<cudaStream_t>(stream);
    return precision == PD_PREC_FP64 ? fma_peak_t<double>(reps, st, tflops) : fma_peak_t<float>(reps, st, tflops);
}

// ---------------------------------------------------------------------------
// Allocation-free multi-dot.  Its partial sums live in the file-scope device
// array below instead of memory obtained from cudaMalloc, so a caller that must
// not allocate device memory (for example one whose host code runs where a
// cudaMalloc/cudaFree, with their implicit device-wide synchronisation, is not
// acceptable, or an application that hands this library no memory beyond the
// buffers it passes) can still use it.  Every GPU that loads the library holds
// the array (kNoAllocScratchDoubles doubles, 524,288 bytes) until the process
// exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxDevices = 64;
constexpr int kNoAllocScratchDoubles = kMaxVecGrid * kMaxWindow;   // one row of kMaxWindow per streaming CTA
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress while that device is current.
int noalloc_scratch(double **out)
{
    int dev = 0;
    PD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(PD_ENOTSUP, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(PD_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
        }
        g_noalloc_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_noalloc_ptr[dev];
    return PD_OK;
}

}  // namespace

int pairdiag_multidot_noalloc(int dtype, const void *Q_dev, int64_t ld, int m, const void *p_dev, int64_t n,
                              double *out_dev, void *stream)
{
    if (!Q_dev || !p_dev || !out_dev) return fail(PD_EINVAL, "null argument");
    if (dtype != 0 && dtype != 1) return fail(PD_EINVAL, "dtype must be 0 (double) or 1 (float)");
    if (m < 1 || m > kMaxWindow)
        return fail(PD_EINVAL, "m=%d outside 1..%d: the static scratch holds partial sums for at most %d vectors",
                    m, kMaxWindow, kMaxWindow);
    if (n < 0 || ld < n) return fail(PD_EINVAL, "need 0 <= n <= ld");
    if ((int64_t)vec_grid() * kMaxWindow > kNoAllocScratchDoubles)
        return fail(PD_ENOTSUP, "streaming grid larger than the static scratch");
    double *scratch = nullptr;
    PD_TRY(noalloc_scratch(&scratch));
    // Every partial sum the reduction reads is written by the same call first,
    // so nothing in the scratch has to start at zero.
    PD_CUDA(multidot_launch(dtype, Q_dev, ld, m, p_dev, n, scratch, out_dev, static_cast<cudaStream_t>(stream)));
    return PD_OK;
}

}  // extern "C"
