// pd_batch.cu -- many pairing Hamiltonians solved together (the mean-field
// use case the paper targets: a pairing solve inside every iteration of a
// self-consistent loop, Sec. 1 and Sec. 6).
//
// All problems run restarted Lanczos in lock step.  One launch per kernel
// serves every problem: the H*x kernel walks the concatenated block list of
// all problems, and the vector kernels work on vectors concatenated over
// problems, cut into chunks that never cross a problem boundary, with
// per-problem coefficients and per-problem reductions.  Each problem carries a
// skip flag (converged, or broken down in the current cycle) that every kernel
// honours, so finished problems cost nothing.  The steps of one restart cycle
// are captured once into a CUDA graph and replayed; the host synchronises once
// per cycle to count the problems still running.
#include "pd_internal.h"
#include "pairdiag.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

using namespace pd;

namespace pd {
// pd_lanczos.cu: after step i of a cycle, problems whose lowest Ritz pair of
// the steps so far meets tol end the cycle (broken and skip set)
cudaError_t batch_ritz_estimate_launch(BatchState *S, int count, int i, double tol, cudaStream_t st);
}

namespace {

struct DevBuf {
    std::vector<void *> ptrs;
    ~DevBuf()
    {
        cudaDeviceSynchronize();                // as cudaFree did: nothing queued still uses them
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
    ~Graph()
    {
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
    }
};

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
    const int dtype = opt.precision == PD_PREC_MIXED ? 1 : 0;

    // ---- validation and host tables ----------------------------------------
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
    int64_t e_off = 0, g_off = 0;
    int max_omega = 1, max_L = 1, max_H = 0, max_block = 1, max_hh = 0;
    for (int p = 0; p < count; ++p) {
        const int om = omega[p], n = n_pairs[p];
        if (om < 1 || om > kMaxOmega || n < 0 || n > om)
            return fail(PD_EINVAL, "batch: problem %d has omega=%d, n_pairs=%d", p, om, n);
        const double *e = e_all + e_off;
        const double *G = G_all + g_off;
        for (int i = 0; i < om; ++i) {
            if (!std::isfinite(e[i])) return fail(PD_EINVAL, "batch: problem %d: e[%d] not finite", p, i);
            for (int j = 0; j < om; ++j) {
                if (!std::isfinite(G[i * om + j])) return fail(PD_EINVAL, "batch: problem %d: G not finite", p);
                if (G[i * om + j] != G[j * om + i]) return fail(PD_EINVAL, "batch: problem %d: G not symmetric", p);
            }
        }
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
            if (bb != run) return fail(PD_ECUDA, "batch: internal block index mismatch (problem %d)", p);
            blk_prob.push_back((uint32_t)p);
            blk_h.push_back(w);
            blk_base.push_back(bb);
            run += host_binom(L, n - __builtin_popcountll(w));
        }
        if ((int64_t)run != dim) return fail(PD_ECUDA, "batch: blocks do not cover problem %d", p);
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
        e_off += om;
        g_off += (int64_t)om * om;
        max_omega = std::max(max_omega, om);
        max_L = std::max(max_L, L);
        max_H = std::max(max_H, H);
    }

    // ---- device data -------------------------------------------------------
    PD_CUDA(cudaGetLastError());
    DevBuf buf;
    BatchDesc *d_desc; uint32_t *d_bp; uint64_t *d_bh, *d_bb, *d_binom;
    uint16_t *d_lw, *d_rk;
    double *d_G64, *d_d64; float *d_G32, *d_d32;
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
    PD_TRY(buf.upload(&d_cp, chunk_prob));
    PD_TRY(buf.upload(&d_cl, chunk_len));
    PD_TRY(buf.upload(&d_cs, chunk_start));
    PD_TRY(buf.upload(&d_pc0, prob_chunk0));
    PD_TRY(buf.upload(&d_pnc, prob_nchunk));
    PD_TRY(buf.upload(&d_po, prob_off));

    BatchBlocks BB{};
    BB.nblocks = (int64_t)blk_prob.size();
    BB.blk_prob = d_bp; BB.blk_h = d_bh; BB.blk_base = d_bb; BB.desc = d_desc;
    BB.lowword_all = d_lw; BB.rankL_all = d_rk; BB.binom = d_binom;
    BB.max_omega = max_omega; BB.max_L = max_L; BB.max_H = max_H; BB.max_block = max_block; BB.max_hh = max_hh;
    BatchVec V{};
    V.count = count; V.nchunks = (int)chunk_prob.size(); V.total = total;
    V.chunk_prob = d_cp; V.chunk_start = d_cs; V.chunk_len = d_cl;
    V.prob_chunk0 = d_pc0; V.prob_nchunk = d_pnc; V.prob_off = d_po;
    HxProblem P{d_G64, d_d64, d_G32, d_d32};

    const int m = std::min(opt.window, kMaxWindow);
    double *part; BatchState *S; int *d_active, *d_counter;
    PD_TRY(buf.alloc(&part, (size_t)V.nchunks * kMaxWindow));
    PD_TRY(buf.alloc(&S, (size_t)count));
    PD_TRY(buf.alloc(&d_active, 1));
    PD_TRY(buf.alloc(&d_counter, 4));
    PD_CUDA(cudaMemsetAsync(S, 0, sizeof(BatchState) * count, st));
    const int *skip = &S[0].skip;
    const int skip_stride = (int)(sizeof(BatchState) / sizeof(int));
    const int sd = (int)(sizeof(BatchState) / sizeof(double));
    cudaEvent_t ev0;
    PD_CUDA(cudaEventCreate(&ev0));
    PD_CUDA(cudaEventRecord(ev0, st));
    std::vector<cudaEvent_t> cyc_ev;             // end of each cycle's convergence test
    std::vector<int> cyc_index;                  // global cycle number of each event
    int cycles = 0;                              // cycles run so far (both phases)

    // Restarted Lanczos for every problem that is not done, on storage type
    // `dt`.  Q_0 of the window holds the start vectors.
    auto run_phase = [&](int dt, char *Q, char *pvc, double tol_run, int stall_check, int max_cycles) -> int {
        const size_t es = dt == 0 ? 8 : 4;
        void *pv = pvc;
        auto q = [&](int j) { return (void *)(Q + es * (size_t)j * (size_t)total); };
        const int hx_grid_ = hx_batch_grid(BB, dt);
        auto step = [&](int i) -> int {
            PD_CUDA(hx_batch_launch(BB, P, dt, q(i), pv, d_counter, hx_grid_, st, skip, skip_stride));
            PD_CUDA(seg_dots_launch(dt, V, q(i), total, 1, pv, S, part, &S[0].c1, sd, st));
            PD_CUDA(seg_recur_project_launch(dt, V, Q, total, i, pv, S, part, st));
            PD_CUDA(seg_update_launch(dt, V, Q, total, i + 1, pv, S, part, st));
            PD_CUDA(batch_finalize_launch(S, count, i, st));
            return PD_OK;
        };
        // steps 1..m-1, the tridiagonal solves, the Ritz vectors and their normalisation
        auto cycle_tail = [&]() -> int {
            for (int i = 1; i < m; ++i) {
                PD_CUDA(seg_scale_launch(dt, V, pv, q(i), S, i - 1, 0, st));
                PD_TRY(step(i));
                // every 4 steps: problems whose Ritz pair meets tol end the cycle
                if ((i + 1) % 4 == 0 && i + 1 < m) PD_CUDA(batch_ritz_estimate_launch(S, count, i, tol_run, st));
            }
            PD_CUDA(batch_tridiag_launch(S, count, st));
            PD_CUDA(seg_ritz_launch(dt, V, Q, total, S, part, st));
            PD_CUDA(seg_scale_launch(dt, V, q(0), q(0), S, 0, 1, st));
            return PD_OK;
        };
        // normalise the start vectors of the open problems
        PD_CUDA(seg_dots_launch(dt, V, q(0), total, 1, q(0), S, part, &S[0].norm2, sd, st));
        PD_CUDA(seg_scale_launch(dt, V, q(0), q(0), S, 0, 1, st));

        // capture the cycle tail once (replayed launches are added to the counter)
        Graph graph;
        long long tail_launches = 0;
        {
            PD_CUDA(cudaStreamSynchronize(st));
            cudaStream_t cs = st;
            bool own = false;
            if (cs == nullptr) {                  // the legacy stream cannot be captured
                PD_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
                own = true;
            }
            const long long before = g_kernel_launches.load();
            cudaStream_t saved = st;
            st = cs;
            PD_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
            const int cap = cycle_tail();
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(st, &g);
            st = saved;
            if (own) cudaStreamDestroy(cs);
            if (cap != PD_OK) { if (g) cudaGraphDestroy(g); return cap; }
            if (ec != cudaSuccess) return fail(PD_ECUDA, "batch: capture failed: %s", cudaGetErrorString(ec));
            graph.g = g;
            PD_CUDA(cudaGraphInstantiate(&graph.ge, g, 0));
            tail_launches = g_kernel_launches.load() - before;
            g_kernel_launches.fetch_sub(tail_launches);   // captured, not yet launched
        }
        int active = count;
        for (int cycle = 0; cycle <= max_cycles; ++cycle) {
            PD_CUDA(batch_reset_launch(S, count, st));
            PD_TRY(step(0));
            PD_CUDA(batch_converge_launch(S, count, tol_run, cycles, stall_check, d_active, st));
            cudaEvent_t ev;
            PD_CUDA(cudaEventCreate(&ev));
            cyc_ev.push_back(ev);
            cyc_index.push_back(cycles);
            PD_CUDA(cudaEventRecord(ev, st));
            PD_CUDA(cudaMemcpyAsync(&active, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
            PD_CUDA(cudaStreamSynchronize(st));
            ++cycles;
            if (active == 0) break;
            PD_CUDA(cudaGraphLaunch(graph.ge, st));
            g_kernel_launches.fetch_add(tail_launches);
        }
        return PD_OK;
    };

    int rc = PD_OK;
    char *Q32 = nullptr, *p32 = nullptr, *Q64 = nullptr, *p64 = nullptr;
    double *v64 = nullptr, *w64 = nullptr;
    rc = [&]() -> int {
        if (dtype == 1) {
            PD_TRY(buf.alloc(&Q32, 4 * (size_t)m * (size_t)total));
            PD_TRY(buf.alloc(&p32, 4 * (size_t)total));
            if (opt.start == PD_START_MLP)
                PD_TRY(batch_mlp_start(mlp, BB, count, omega, n_pairs, e_all, G_all, 1, Q32, st));
            else
                PD_CUDA(seg_random_launch(1, V, Q32, opt.seed, st));
            // FP32 cycles aim a little below tol so that the FP64 residual of the
            // refined vector, which also carries the FP32 rounding, stays within tol
            PD_TRY(run_phase(1, Q32, p32, std::max(0.5 * tol, opt.mixed_floor), 1, opt.max_restarts));
            // FP64 Rayleigh refinement of every problem
            PD_TRY(buf.alloc(&v64, (size_t)total));
            PD_TRY(buf.alloc(&w64, (size_t)total));
            PD_CUDA(convert_launch(0, v64, 1, Q32, total, st));
            PD_CUDA(hx_batch_launch(BB, P, 0, v64, w64, d_counter, hx_batch_grid(BB, 0), st, nullptr, 0));
            PD_CUDA(seg_dots_launch(0, V, v64, total, 1, w64, nullptr, part, &S[0].c2[0], sd, st));
            PD_CUDA(seg_dots_launch(0, V, v64, total, 1, v64, nullptr, part, &S[0].c2[1], sd, st));
            PD_CUDA(batch_rayleigh_launch(S, count, 0, st));
            PD_CUDA(seg_residual_launch(V, w64, v64, S, part, st));
            PD_CUDA(batch_rayleigh_launch(S, count, 1, st));
            // problems whose FP64 residual misses tol continue in FP64 from the refined vector
            int reopened = 0;
            PD_CUDA(batch_reopen_launch(S, count, tol, cycles - 1, d_active, st));
            PD_CUDA(cudaMemcpyAsync(&reopened, d_active, sizeof(int), cudaMemcpyDeviceToHost, st));
            PD_CUDA(cudaStreamSynchronize(st));
            if (reopened > 0) {
                PD_TRY(buf.alloc(&Q64, 8 * (size_t)m * (size_t)total));
                PD_TRY(buf.alloc(&p64, 8 * (size_t)total));
                PD_CUDA(cudaMemcpyAsync(Q64, v64, 8 * (size_t)total, cudaMemcpyDeviceToDevice, st));
                const int left = std::max(0, opt.max_restarts - cycles);
                PD_TRY(run_phase(0, Q64, p64, tol, 0, left));
            }
        } else {
            PD_TRY(buf.alloc(&Q64, 8 * (size_t)m * (size_t)total));
            PD_TRY(buf.alloc(&p64, 8 * (size_t)total));
            if (opt.start == PD_START_MLP)
                PD_TRY(batch_mlp_start(mlp, BB, count, omega, n_pairs, e_all, G_all, 0, Q64, st));
            else
                PD_CUDA(seg_random_launch(0, V, Q64, opt.seed, st));
            PD_TRY(run_phase(0, Q64, p64, tol, 0, opt.max_restarts));
        }
        return PD_OK;
    }();

    // ---- results -------------------------------------------------------------
    std::vector<BatchState> hs(count);
    if (rc == PD_OK) {
        const cudaError_t e1 = cudaMemcpyAsync(hs.data(), S, sizeof(BatchState) * count, cudaMemcpyDeviceToHost, st);
        const cudaError_t e2 = cudaStreamSynchronize(st);
        if (e1 != cudaSuccess || e2 != cudaSuccess) rc = fail(PD_ECUDA, "batch: result copy failed");
    }
    std::vector<float> cyc_ms(cycles, 0.0f);
    for (size_t c = 0; c < cyc_ev.size(); ++c) {
        if (rc == PD_OK) cudaEventElapsedTime(&cyc_ms[cyc_index[c]], ev0, cyc_ev[c]);
        cudaEventDestroy(cyc_ev[c]);
    }
    cudaEventDestroy(ev0);
    if (rc != PD_OK) return rc;
    int nfail = 0;
    for (int p = 0; p < count; ++p) {
        const BatchState &B = hs[p];
        e0[p] = B.e0;
        const bool ok = B.done && std::isfinite(B.e0) && B.rel <= tol;
        status[p] = ok ? PD_OK : PD_ENOCONV;
        if (!ok) ++nfail;
        if (results) {
            results[p].iterations = B.iters;
            results[p].converged = ok ? 1 : 0;
            results[p].stalled = B.stalled;
            results[p].rel_residual = B.rel;
            const int c = B.done ? B.done_cycle : cycles - 1;
            results[p].latency_ms = (c >= 0 && c < cycles) ? cyc_ms[c] : 0.0;
        }
    }
    if (nfail) return fail(PD_ENOCONV, "batch: %d of %d problems did not reach tol %.3g", nfail, count, tol);
    return PD_OK;
}
