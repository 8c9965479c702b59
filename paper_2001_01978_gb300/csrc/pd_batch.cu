// pd_batch.cu -- many pairing Hamiltonians solved together (the mean-field
// use case the paper targets: a pairing solve inside every iteration of a
// self-consistent loop, Sec. 1 and Sec. 6).
//
// Size classes.  The problems are sorted by dimension and cut into up to four
// classes (the smallest half, the next 30 %, 15 % and the largest 5 %).  Each
// class runs on a stream of its own, and the smaller classes at a higher
// stream priority, so a class of small problems finishes as soon as its own
// problems do instead of waiting, iteration by iteration, for the largest
// problems of the call.
//
// Within a class all problems run restarted Lanczos in lock step.  One launch
// per kernel serves every problem of the class: the H*x kernel walks the
// concatenated block list of its problems, and the vector kernels work on
// vectors concatenated over problems, cut into chunks that never cross a
// problem boundary, with per-problem coefficients and per-problem reductions.
// Each problem carries a skip flag (converged, or broken down in the current
// cycle) that every kernel honours, so finished problems cost nothing.
//
// Device-side cycle loop.  The restart cycles of a class are one CUDA graph:
// a prologue (normalised start vectors, the first Lanczos step and the
// convergence test of the first cycle) and a conditional WHILE node whose body
// is one cycle (the rest of the cycle's steps, the tridiagonal solves and
// Ritz vectors, then the next cycle's first step and convergence test).  A
// one-thread kernel at the end of each body sets the loop condition on the
// device: problems still running and cycles left.  The host does not
// synchronise between cycles; the FP64 form synchronises once, at the end,
// and the mixed form once more, after the FP64 refinement, to see whether any
// problem needs FP64 cycles.
#include "pd_internal.h"
#include "pairdiag.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <numeric>
#include <vector>

using namespace pd;

namespace pd {
// pd_lanczos.cu: after step i of a cycle, problems whose lowest Ritz pair of
// the steps so far meets tol end the cycle (broken and skip set)
cudaError_t batch_ritz_estimate_launch(BatchState *S, int count, int i, double tol, cudaStream_t st);
}

namespace {

constexpr int kMaxClasses = 4;

struct DevBuf {
    std::vector<void *> ptrs;
    cudaStream_t st = nullptr;           // the stream that used the blocks
    ~DevBuf()
    {
        // no queued work may still use them (the cache hands them out again)
        if (!ptrs.empty()) cudaStreamSynchronize(st);
        for (void *p : ptrs) pool_free(p);
    }
    template <typename T>
    int alloc(T **p, size_t count)
    {
        void *q = nullptr;
        const cudaError_t e = pool_alloc(&q, std::max<size_t>(16, count * sizeof(T)));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(PD_ENOMEM, "batch: cudaMalloc(%zu bytes): %s", count * sizeof(T), cudaGetErrorString(e));
        }
        ptrs.push_back(q);
        *p = static_cast<T *>(q);
        return PD_OK;
    }
    template <typename T>
    int upload(T **p, const std::vector<T> &v)
    {
        PD_TRY(alloc(p, v.size()));
        PD_CUDA(cudaMemcpy(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return PD_OK;
    }
};

struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    long long prologue_launches = 0;     // kernels of the prologue
    long long body_launches = 0;         // kernels of one loop iteration
    ~Graph()
    {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    }
};

// A stream the class may own; destroyed after every other member of the class
struct ClassStream {
    cudaStream_t st = nullptr;
    bool own = false;
    ~ClassStream()
    {
        if (own && st) cudaStreamDestroy(st);
    }
};

// One size class: its problems, tables, buffers, stream and graphs.  Members
// are destroyed in reverse order: the buffers first (after a synchronisation
// of the class's stream), the stream last.
struct ClassRun {
    ClassStream cs;
    cudaStream_t &st = cs.st;
    std::vector<int> prob;               // indices into the caller's arrays
    int count = 0;
    BatchBlocks BB{};
    BatchVec V{};
    HxProblem P{};
    int64_t total = 0;
    std::vector<int> omega, n_pairs;     // of the class's problems
    std::vector<double> e_all, G_all;
    BatchState *S = nullptr;
    double *part = nullptr;
    int *ctl = nullptr;                  // [0] running problems, [1] cycle number, [2] reopened
    unsigned long long *counter = nullptr;   // [0] next block, [1] finished CTAs of the batched H*x
    char *Q32 = nullptr, *p32 = nullptr, *Q64 = nullptr, *p64 = nullptr;
    double *v64 = nullptr, *w64 = nullptr;
    Graph phase[2];                      // 0: FP32 (mixed) or FP64 phase, 1: FP64 continuation
    int reopened = 0;
    DevBuf buf;                          // destroyed first (declared last): syncs st
};

// Host tables and device buffers of one class.
int setup_class(ClassRun &c, const pairdiag_options &opt, const int *omega, const int *n_pairs,
                const std::vector<int64_t> &e_off, const std::vector<int64_t> &g_off, const double *e_all,
                const double *G_all)
{
    const int count = c.count;
    std::vector<BatchDesc> desc(count);
    std::vector<uint32_t> blk_prob;
    std::vector<uint64_t> blk_h, blk_base;
    std::vector<double> G64, d64;
    std::vector<float> G32, d32;
    std::map<int, int> tab_of_L;
    std::vector<uint16_t> lowword_all, rankL_all;
    std::vector<int> chunk_prob, chunk_len, prob_chunk0, prob_nchunk;
    std::vector<int64_t> chunk_start, prob_off;
    int64_t total = 0;
    int max_omega = 1, max_L = 1, max_H = 0, max_block = 1, max_hh = 0, max_n = 0;
    for (int p = 0; p < count; ++p) {
        const int q = c.prob[p];
        const int om = omega[q], n = n_pairs[q];
        const double *e = e_all + e_off[q];
        const double *G = G_all + g_off[q];
        c.omega.push_back(om);
        c.n_pairs.push_back(n);
        c.e_all.insert(c.e_all.end(), e, e + om);
        c.G_all.insert(c.G_all.end(), G, G + (size_t)om * om);
        int L = opt.low_bits > 0 ? opt.low_bits : 12;
        if (opt.low_bits == 0) {                  // an autotuned block split for this (omega, N)
            int lb = 0, hv = 0;
            if (pairdiag_tune_get(om, n, opt.precision, &lb, &hv) == PD_OK && lb > 0) L = lb;
        }
        L = std::min(L, std::min(om, kMaxLow));
        const int H = om - L;
        if (!tab_of_L.count(L)) {
            tab_of_L[L] = (int)lowword_all.size();
            const int nL = 1 << L;
            std::vector<int> off(L + 2, 0), fill(L + 2, 0);
            for (int k = 0; k <= L; ++k) off[k + 1] = off[k] + (int)host_binom(L, k);
            lowword_all.resize(lowword_all.size() + nL);
            rankL_all.resize(rankL_all.size() + nL);
            const int base = tab_of_L[L];
            for (int w = 0; w < nL; ++w) {
                const int k = __builtin_popcount(w);
                rankL_all[base + w] = (uint16_t)fill[k];
                lowword_all[base + off[k] + fill[k]] = (uint16_t)w;
                ++fill[k];
            }
        }
        const int64_t dim = (int64_t)host_binom(om, n);
        max_n = std::max(max_n, n);
        BatchDesc &D = desc[p];
        D.omega = om; D.n = n; D.L = L;
        D.g_off = (int)G64.size(); D.d_off = (int)d64.size();
        D.tab_off = tab_of_L[L];
        D.vec_off = total; D.dim = dim;
        for (int i = 0; i < om * om; ++i) { G64.push_back(G[i]); G32.push_back((float)G[i]); }
        for (int i = 0; i < om; ++i) {
            const double dv = 2.0 * e[i] + G[i * om + i];
            d64.push_back(dv);
            d32.push_back((float)dv);
        }
        // blocks of this problem
        const int kmin = std::max(0, n - H), kmax = std::min(n, L);
        std::vector<uint64_t> hw;
        for (int k = kmin; k <= kmax; ++k) {
            words_with_popcount(H, n - k, hw);
            max_block = std::max(max_block, (int)host_binom(L, k));
            max_hh = std::max(max_hh, (n - k) * (H - (n - k)));
        }
        std::sort(hw.begin(), hw.end());
        uint64_t run = 0;
        for (uint64_t w : hw) {
            const uint64_t bb = host_block_base(w, L, n);
            if (bb != run) return fail(PD_ECUDA, "batch: internal block index mismatch (problem %d)", q);
            blk_prob.push_back((uint32_t)p);
            blk_h.push_back(w);
            blk_base.push_back(bb);
            run += host_binom(L, n - __builtin_popcountll(w));
        }
        if ((int64_t)run != dim) return fail(PD_ECUDA, "batch: blocks do not cover problem %d", q);
        // chunks: at most 32 per problem, at least ~1024 elements each, each a
        // multiple of 4 elements long (but the last), so that every chunk starts
        // on a 16-byte boundary (problems start on one: see total below)
        const int nc = (int)std::min<int64_t>(kMaxChunksPerProblem, std::max<int64_t>(1, (dim + 1023) / 1024));
        const int64_t clen = ((dim + nc - 1) / nc + 3) & ~int64_t(3);
        prob_chunk0.push_back((int)chunk_prob.size());
        int made = 0;
        for (int64_t s0 = 0; s0 < dim; s0 += clen, ++made) {
            chunk_prob.push_back(p);
            chunk_start.push_back(total + s0);
            chunk_len.push_back((int)std::min<int64_t>(clen, dim - s0));
        }
        prob_nchunk.push_back(made);
        prob_off.push_back(total);
        total += (dim + 3) & ~int64_t(3);     // next problem on a 4-element boundary
        max_omega = std::max(max_omega, om);
        max_L = std::max(max_L, L);
        max_H = std::max(max_H, H);
    }

    DevBuf &buf = c.buf;
    buf.st = c.st;
    BatchDesc *d_desc; uint32_t *d_bp; uint64_t *d_bh, *d_bb, *d_binom;
    uint16_t *d_lw, *d_rk;
    double *d_G64, *d_d64; float *d_G32, *d_d32; float2 *d_Gff, *d_dff;
    int *d_cp, *d_cl, *d_pc0, *d_pnc; int64_t *d_cs, *d_po;
    std::vector<uint64_t> binom(64 * 64);
    for (int i = 0; i < 64; ++i)
        for (int j = 0; j < 64; ++j) binom[i * 64 + j] = host_binom(i, j);
    PD_TRY(buf.upload(&d_desc, desc));
    PD_TRY(buf.upload(&d_bp, blk_prob));
    PD_TRY(buf.upload(&d_bh, blk_h));
    PD_TRY(buf.upload(&d_bb, blk_base));
    PD_TRY(buf.upload(&d_binom, binom));
    PD_TRY(buf.upload(&d_lw, lowword_all));
    PD_TRY(buf.upload(&d_rk, rankL_all));
    PD_TRY(buf.upload(&d_G64, G64));
    PD_TRY(buf.upload(&d_d64, d64));
    PD_TRY(buf.upload(&d_G32, G32));
    PD_TRY(buf.upload(&d_d32, d32));
    {   // G and d split into two FP32 parts: the float-float refinement product
        auto split = [](const std::vector<double> &v) {
            std::vector<float2> r(v.size());
            for (size_t i = 0; i < v.size(); ++i) {
                const float hi = (float)v[i];
                r[i] = make_float2(hi, (float)(v[i] - (double)hi));
            }
            return r;
        };
        PD_TRY(buf.upload(&d_Gff, split(G64)));
        PD_TRY(buf.upload(&d_dff, split(d64)));
    }
    PD_TRY(buf.upload(&d_cp, chunk_prob));
    PD_TRY(buf.upload(&d_cl, chunk_len));
    PD_TRY(buf.upload(&d_cs, chunk_start));
    PD_TRY(buf.upload(&d_pc0, prob_chunk0));
    PD_TRY(buf.upload(&d_pnc, prob_nchunk));
    PD_TRY(buf.upload(&d_po, prob_off));

    BatchBlocks &BB = c.BB;
    BB.nblocks = (int64_t)blk_prob.size();
    BB.blk_prob = d_bp; BB.blk_h = d_bh; BB.blk_base = d_bb; BB.desc = d_desc;
    BB.lowword_all = d_lw; BB.rankL_all = d_rk; BB.binom = d_binom;
    BB.max_omega = max_omega; BB.max_L = max_L; BB.max_H = max_H; BB.max_block = max_block; BB.max_hh = max_hh;
    BB.max_n = max_n;
    // the batched H*x: direct gathers (variant 3) unless the caller asks for the staged form
    BB.variant = (opt.hx_variant == 1 || opt.hx_variant == 2) ? 1 : 3;
    BatchVec &V = c.V;
    V.count = count; V.nchunks = (int)chunk_prob.size(); V.total = total;
    V.chunk_prob = d_cp; V.chunk_start = d_cs; V.chunk_len = d_cl;
    V.prob_chunk0 = d_pc0; V.prob_nchunk = d_pnc; V.prob_off = d_po;
    c.P = HxProblem{d_G64, d_d64, d_G32, d_d32, d_Gff, d_dff};
    c.total = total;

    PD_TRY(buf.alloc(&c.part, (size_t)V.nchunks * kMaxWindow));
    PD_TRY(buf.alloc(&c.S, (size_t)count));
    PD_TRY(buf.alloc(&c.ctl, 4));
    PD_TRY(buf.alloc(&c.counter, 2));
    PD_CUDA(cudaMemsetAsync(c.S, 0, sizeof(BatchState) * count, c.st));
    PD_CUDA(cudaMemsetAsync(c.ctl, 0, sizeof(int) * 4, c.st));
    PD_CUDA(cudaMemsetAsync(c.counter, 0, sizeof(unsigned long long) * 2, c.st));
    return PD_OK;
}

// Restarted Lanczos of every problem of the class that is not done, on storage
// type dt, as one graph: prologue + WHILE(cycle).  Q_0 of the window holds the
// start vectors.  The graph is built here and launched on the class's stream.
int build_phase_graph(ClassRun &c, int dt, int window, char *Q, char *pvc, double tol_run, int stall_check,
                      int max_cycles, Graph &gr)
{
    const int count = c.count;
    const int m = std::min(window, kMaxWindow);
    const size_t es = dt == 0 ? 8 : 4;
    const int64_t total = c.total;
    const BatchVec &V = c.V;
    const BatchBlocks &BB = c.BB;
    BatchState *S = c.S;
    double *part = c.part;
    void *pv = pvc;
    const int *skip = &S[0].skip;
    const int skip_stride = (int)(sizeof(BatchState) / sizeof(int));
    const int sd = (int)(sizeof(BatchState) / sizeof(double));
    auto q = [&](int j) { return (void *)(Q + es * (size_t)j * (size_t)total); };
    const int hx_grid_ = hx_batch_grid(BB, dt);
    cudaStream_t cs = nullptr;                    // the capturing stream
    auto step = [&](int i) -> int {
        PD_CUDA(hx_batch_launch(BB, c.P, dt, q(i), pv, c.counter, hx_grid_, cs, skip, skip_stride));
        PD_CUDA(seg_dots_launch(dt, V, q(i), total, 1, pv, S, part, &S[0].c1, sd, cs));
        PD_CUDA(seg_recur_project_launch(dt, V, Q, total, i, pv, S, part, cs));
        PD_CUDA(seg_update_launch(dt, V, Q, total, i + 1, pv, S, part, cs));
        PD_CUDA(batch_finalize_launch(S, count, i, cs));
        return PD_OK;
    };
    // a cycle's first step and its convergence test, then the loop condition
    auto head = [&](cudaGraphConditionalHandle loop) -> int {
        PD_CUDA(batch_reset_launch(S, count, cs));
        PD_TRY(step(0));
        PD_CUDA(batch_converge_launch(S, count, tol_run, &c.ctl[1], stall_check, &c.ctl[0], cs));
        PD_CUDA(batch_ctl_launch(c.ctl, max_cycles, loop, cs));
        return PD_OK;
    };
    // steps 1..m-1, the tridiagonal solves, the Ritz vectors and their normalisation
    auto tail = [&]() -> int {
        for (int i = 1; i < m; ++i) {
            PD_CUDA(seg_scale_launch(dt, V, pv, q(i), S, i - 1, 0, cs));
            PD_TRY(step(i));
            // every 4 steps: problems whose Ritz pair meets tol end the cycle
            if ((i + 1) % 4 == 0 && i + 1 < m) PD_CUDA(batch_ritz_estimate_launch(S, count, i, tol_run, cs));
        }
        PD_CUDA(batch_tridiag_launch(S, count, cs));
        PD_CUDA(seg_ritz_launch(dt, V, Q, total, S, part, cs));
        PD_CUDA(seg_scale_launch(dt, V, q(0), q(0), S, 0, 1, cs));
        return PD_OK;
    };

    PD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    const int rc = [&]() -> int {
        PD_CUDA(cudaGraphCreate(&gr.g, 0));
        cudaGraphConditionalHandle loop;
        PD_CUDA(cudaGraphConditionalHandleCreate(&loop, gr.g, 0, 0));
        // prologue: normalise the start vectors of the open problems, first cycle head
        const long long l0 = g_kernel_launches.load();
        PD_CUDA(cudaStreamBeginCaptureToGraph(cs, gr.g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        int r = [&]() -> int {
            PD_CUDA(seg_dots_launch(dt, V, q(0), total, 1, q(0), S, part, &S[0].norm2, sd, cs));
            PD_CUDA(seg_scale_launch(dt, V, q(0), q(0), S, 0, 1, cs));
            PD_TRY(head(loop));
            return PD_OK;
        }();
        cudaStreamCaptureStatus cst;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        std::vector<cudaGraphNode_t> last;
        if (r == PD_OK) {
            const cudaError_t e = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
            if (e != cudaSuccess) r = fail(PD_ECUDA, "batch: capture info: %s", cudaGetErrorString(e));
            else last.assign(deps, deps + ndeps);
        }
        cudaGraph_t cap = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &cap);
        if (r != PD_OK) return r;
        if (ec != cudaSuccess) return fail(PD_ECUDA, "batch: prologue capture: %s", cudaGetErrorString(ec));
        gr.prologue_launches = g_kernel_launches.load() - l0;
        // the loop: WHILE(condition set by the last kernel of the prologue / body)
        cudaGraphNodeParams cp{};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = loop;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t wnode;
        PD_CUDA(cudaGraphAddNode(&wnode, gr.g, last.data(), nullptr, last.size(), &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        const long long l1 = g_kernel_launches.load();
        PD_CUDA(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
        r = [&]() -> int {
            PD_TRY(tail());
            PD_TRY(head(loop));
            return PD_OK;
        }();
        cudaGraph_t bcap = nullptr;
        const cudaError_t eb = cudaStreamEndCapture(cs, &bcap);
        if (r != PD_OK) return r;
        if (eb != cudaSuccess) return fail(PD_ECUDA, "batch: loop body capture: %s", cudaGetErrorString(eb));
        gr.body_launches = g_kernel_launches.load() - l1;
        PD_CUDA(cudaGraphInstantiate(&gr.ge, gr.g, 0));
        return PD_OK;
    }();
    // captured, not launched: the launches are counted when the graph runs
    g_kernel_launches.fetch_sub(gr.prologue_launches + gr.body_launches);
    cudaStreamDestroy(cs);
    return rc;
}

// Buffers, start vectors and the first phase's graph of one class.  Done for
// every class before any graph runs: the network pass of the learned start
// frees memory, which would wait for work already running on the device.
int prepare_class(ClassRun &c, const pairdiag_options &opt, pairdiag_mlp *mlp, double tol)
{
    const int m = std::min(opt.window, kMaxWindow);
    const int dtype = opt.precision == PD_PREC_MIXED ? 1 : 0;
    const int64_t total = c.total;
    cudaStream_t st = c.st;
    DevBuf &buf = c.buf;
    char *&Q = dtype == 1 ? c.Q32 : c.Q64;
    char *&pv = dtype == 1 ? c.p32 : c.p64;
    const size_t es = dtype == 1 ? 4 : 8;
    PD_TRY(buf.alloc(&Q, es * (size_t)m * (size_t)total));
    PD_TRY(buf.alloc(&pv, es * (size_t)total));
    if (dtype == 1) {
        PD_TRY(buf.alloc(&c.v64, (size_t)total));
        PD_TRY(buf.alloc(&c.w64, (size_t)total));
    }
    if (opt.start == PD_START_MLP)
        PD_TRY(batch_mlp_start(mlp, c.BB, c.count, c.omega.data(), c.n_pairs.data(), c.e_all.data(), c.G_all.data(),
                               dtype, Q, st));
    else
        PD_CUDA(seg_random_launch(dtype, c.V, Q, opt.seed, st));
    // FP32 cycles aim a little below tol so that the FP64 residual of the
    // refined vector, which also carries the FP32 rounding, stays within tol
    const double tol_run = dtype == 1 ? std::max(0.5 * tol, opt.mixed_floor) : tol;
    PD_TRY(build_phase_graph(c, dtype, m, Q, pv, tol_run, dtype == 1 ? 1 : 0, opt.max_restarts, c.phase[0]));
    int zero = 0;
    PD_CUDA(cudaMemcpyAsync(&c.ctl[1], &zero, sizeof(int), cudaMemcpyHostToDevice, st));
    PD_CUDA(cudaStreamSynchronize(st));
    return PD_OK;
}

// The first phase of one class (the FP32 cycles and the FP64 refinement of the
// mixed form, or the whole FP64 solve), enqueued without a host synchronisation.
int launch_class(ClassRun &c, const pairdiag_options &opt, double tol)
{
    cudaStream_t st = c.st;
    PD_CUDA(cudaGraphLaunch(c.phase[0].ge, st));
    if (opt.precision != PD_PREC_MIXED) return PD_OK;
    // FP64 Rayleigh refinement of every problem
    const int64_t total = c.total;
    const int sd = (int)(sizeof(BatchState) / sizeof(double));
    PD_CUDA(convert_launch(0, c.v64, 1, c.Q32, total, st));
    // w = H v: float-float rows of the FP32 restart vectors where the kernel
    // fits (FP64-accurate, on the FP32 pipes), else FP64 rows of v64
    const int ffg = hx_batch_grid(c.BB, 2);
    if (ffg > 0) PD_CUDA(hx_batch_launch(c.BB, c.P, 2, c.Q32, c.w64, c.counter, ffg, st, nullptr, 0));
    else PD_CUDA(hx_batch_launch(c.BB, c.P, 0, c.v64, c.w64, c.counter, hx_batch_grid(c.BB, 0), st, nullptr, 0));
    PD_CUDA(seg_dots_launch(0, c.V, c.v64, total, 1, c.w64, nullptr, c.part, &c.S[0].c2[0], sd, st));
    PD_CUDA(seg_dots_launch(0, c.V, c.v64, total, 1, c.v64, nullptr, c.part, &c.S[0].c2[1], sd, st));
    PD_CUDA(batch_rayleigh_launch(c.S, c.count, 0, st));
    PD_CUDA(seg_residual_launch(c.V, c.w64, c.v64, c.S, c.part, st));
    PD_CUDA(batch_rayleigh_launch(c.S, c.count, 1, st));
    // problems whose FP64 residual misses tol reopen (counted in ctl[2])
    PD_CUDA(batch_reopen_launch(c.S, c.count, tol, &c.ctl[1], &c.ctl[2], st));
    return PD_OK;
}

// Mixed form, after the refinement: FP64 cycles for the reopened problems.
int continue_class(ClassRun &c, const pairdiag_options &opt, double tol)
{
    int ctl[3] = {0, 0, 0};
    PD_CUDA(cudaMemcpyAsync(ctl, c.ctl, sizeof ctl, cudaMemcpyDeviceToHost, c.st));
    PD_CUDA(cudaStreamSynchronize(c.st));
    c.reopened = ctl[2];
    if (c.reopened == 0) return PD_OK;
    const int m = std::min(opt.window, kMaxWindow);
    PD_TRY(c.buf.alloc(&c.Q64, 8 * (size_t)m * (size_t)c.total));
    PD_TRY(c.buf.alloc(&c.p64, 8 * (size_t)c.total));
    PD_CUDA(cudaMemcpyAsync(c.Q64, c.v64, 8 * (size_t)c.total, cudaMemcpyDeviceToDevice, c.st));
    const int left = std::max(0, opt.max_restarts - ctl[1]);
    PD_TRY(build_phase_graph(c, 0, m, c.Q64, c.p64, tol, 0, left, c.phase[1]));
    PD_CUDA(cudaGraphLaunch(c.phase[1].ge, c.st));   // ctl[1] continues from the FP32 cycles
    return PD_OK;
}

}  // namespace

extern "C" int pairdiag_batch_ground_state(int count, const int *omega, const int *n_pairs, const double *e_all,
                                           const double *G_all, double tol, const pairdiag_options *opt_in,
                                           pairdiag_mlp_t *mlp, double *e0, int *status,
                                           pairdiag_batch_result *results, void *stream)
{
    if (count < 1 || !omega || !n_pairs || !e_all || !G_all || !e0 || !status)
        return fail(PD_EINVAL, "batch: bad argument");
    if (!(tol >= 0.0)) return fail(PD_EINVAL, "batch: tol must be >= 0");
    pairdiag_options opt;
    pairdiag_default_options(&opt);
    if (opt_in) opt = *opt_in;
    if (opt.window < 1 || opt.window > kMaxWindow) return fail(PD_EINVAL, "batch: window outside 1..%d", kMaxWindow);
    if (opt.precision != PD_PREC_FP64 && opt.precision != PD_PREC_MIXED) return fail(PD_EINVAL, "batch: bad precision");
    if (opt.mode != 0) return fail(PD_ENOTSUP, "batch: only the restarted mode is supported");
    if (opt.start != PD_START_RANDOM && opt.start != PD_START_MLP)
        return fail(PD_ENOTSUP, "batch: the start must be PD_START_RANDOM or PD_START_MLP");
    if (opt.start == PD_START_MLP && !mlp) return fail(PD_EINVAL, "batch: PD_START_MLP needs a network");
    if (opt.low_bits < 0 || opt.low_bits > kMaxLow) return fail(PD_EINVAL, "batch: low_bits outside 0..%d", kMaxLow);
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // ---- validation ------------------------------------------------------------
    std::vector<int64_t> e_off(count), g_off(count), dims(count);
    int64_t eo = 0, go = 0;
    for (int p = 0; p < count; ++p) {
        const int om = omega[p], n = n_pairs[p];
        if (om < 1 || om > kMaxOmega || n < 0 || n > om)
            return fail(PD_EINVAL, "batch: problem %d has omega=%d, n_pairs=%d", p, om, n);
        const double *e = e_all + eo;
        const double *G = G_all + go;
        for (int i = 0; i < om; ++i) {
            if (!std::isfinite(e[i])) return fail(PD_EINVAL, "batch: problem %d: e[%d] not finite", p, i);
            for (int j = 0; j < om; ++j) {
                if (!std::isfinite(G[i * om + j])) return fail(PD_EINVAL, "batch: problem %d: G not finite", p);
                if (G[i * om + j] != G[j * om + i]) return fail(PD_EINVAL, "batch: problem %d: G not symmetric", p);
            }
        }
        e_off[p] = eo;
        g_off[p] = go;
        dims[p] = (int64_t)host_binom(om, n);
        eo += om;
        go += (int64_t)om * om;
    }
    PD_CUDA(cudaGetLastError());

    // ---- size classes ------------------------------------------------------------
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dims[a] < dims[b]; });
    const double cuts[kMaxClasses] = {0.50, 0.80, 0.95, 1.0};
    const int nclass = count >= 64 ? kMaxClasses : 1;
    std::vector<std::unique_ptr<ClassRun>> cls;
    int lo = 0;
    for (int k = 0; k < nclass; ++k) {
        const int hi = (k == nclass - 1) ? count : std::max(lo, (int)std::lround(cuts[k] * count));
        if (hi <= lo) continue;
        auto c = std::make_unique<ClassRun>();
        c->prob.assign(order.begin() + lo, order.begin() + hi);
        c->count = hi - lo;
        cls.push_back(std::move(c));
        lo = hi;
    }
    // streams: the smaller classes at a higher priority; every class stream
    // starts after the work already queued on the caller's stream
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    cudaEvent_t ev_start = nullptr;
    PD_CUDA(cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
    unsigned long long *d_t0 = nullptr;
    DevBuf tbuf;
    tbuf.st = st;
    int rc = [&]() -> int {
        PD_TRY(tbuf.alloc(&d_t0, 1));
        PD_CUDA(device_clock_launch(d_t0, st));             // the call's start on the device clock
        PD_CUDA(cudaEventRecord(ev_start, st));
        const int ncls = (int)cls.size();
        for (int k = 0; k < ncls; ++k) {
            ClassRun &c = *cls[k];
            if (ncls == 1) {
                c.st = st;
            } else {
                const int prio = std::max(prio_hi, prio_lo - (ncls - 1 - k));    // smaller class: higher priority
                PD_CUDA(cudaStreamCreateWithPriority(&c.cs.st, cudaStreamNonBlocking, prio));
                c.cs.own = true;
                PD_CUDA(cudaStreamWaitEvent(c.st, ev_start, 0));
            }
            PD_TRY(setup_class(c, opt, omega, n_pairs, e_off, g_off, e_all, G_all));
        }
        for (auto &c : cls) PD_TRY(prepare_class(*c, opt, mlp, tol));
        for (auto &c : cls) PD_TRY(launch_class(*c, opt, tol));
        if (opt.precision == PD_PREC_MIXED)
            for (auto &c : cls) PD_TRY(continue_class(*c, opt, tol));
        for (auto &c : cls) PD_CUDA(cudaStreamSynchronize(c->st));
        return PD_OK;
    }();
    cudaEventDestroy(ev_start);

    // ---- results -----------------------------------------------------------------
    unsigned long long t0 = 0;
    if (rc == PD_OK) {
        const cudaError_t e1 = cudaMemcpy(&t0, d_t0, sizeof t0, cudaMemcpyDeviceToHost);
        if (e1 != cudaSuccess) rc = fail(PD_ECUDA, "batch: clock copy failed");
    }
    int nfail = 0;
    for (auto &cp : cls) {
        if (rc != PD_OK) break;
        ClassRun &c = *cp;
        std::vector<BatchState> hs(c.count);
        int ctl[3] = {0, 0, 0};
        cudaError_t e1 = cudaMemcpyAsync(hs.data(), c.S, sizeof(BatchState) * c.count, cudaMemcpyDeviceToHost, c.st);
        if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(ctl, c.ctl, sizeof ctl, cudaMemcpyDeviceToHost, c.st);
        if (e1 == cudaSuccess) e1 = cudaStreamSynchronize(c.st);
        if (e1 != cudaSuccess) {
            rc = fail(PD_ECUDA, "batch: result copy failed: %s", cudaGetErrorString(e1));
            break;
        }
        // kernels that ran: both graphs' prologues and every executed loop body
        // (ctl[1] counts the cycle heads: one in each prologue, one per body)
        long long ran = 0;
        int heads = ctl[1];
        for (const Graph &g : c.phase) {
            if (!g.ge) continue;
            ran += g.prologue_launches;
            heads -= 1;
        }
        const long long body = c.phase[0].body_launches;
        ran += (long long)std::max(0, heads) * body;
        g_kernel_launches.fetch_add(ran);
        for (int j = 0; j < c.count; ++j) {
            const int p = c.prob[j];
            const BatchState &B = hs[j];
            e0[p] = B.e0;
            const bool ok = B.done && std::isfinite(B.e0) && B.rel <= tol;
            status[p] = ok ? PD_OK : PD_ENOCONV;
            if (!ok) ++nfail;
            if (results) {
                results[p].iterations = B.iters;
                results[p].converged = ok ? 1 : 0;
                results[p].stalled = B.stalled;
                results[p].rel_residual = B.rel;
                results[p].latency_ms = (B.t_done > t0) ? (double)(B.t_done - t0) * 1e-6 : 0.0;
            }
        }
    }
    cls.clear();                                  // syncs and returns every block to the cache
    if (rc != PD_OK) return rc;
    if (nfail) return fail(PD_ENOCONV, "batch: %d of %d problems did not reach tol %.3g", nfail, count, tol);
    return PD_OK;
}
