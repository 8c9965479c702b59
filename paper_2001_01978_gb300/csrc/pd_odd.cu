// pd_odd.cu -- odd-mass systems in the blocking approximation (Eq. 3).
//
// One unpaired particle in orbit b keeps every pair out of b, so the
// seniority-one subspace with b blocked is the seniority-zero space of the
// pairs on the other Omega-1 orbits, and H_b there is the constant e_b plus
// Eq. 2 restricted to those orbits.  Each subspace is therefore an ordinary
// handle of this library on the reduced (e, G): the same basis tables, H*x
// kernels and Lanczos run unchanged.  Block = 0 of the paper (block = -1
// here) needs every b.  Subspaces too small to fill the GPU on their own
// (dim <= 2^17) are solved together by the batched solver (pd_batch.cu) and,
// when the caller wants the winner's vector or occupations, the winning
// subspace once more as a handle.  Larger subspaces are handles solved by up
// to three host threads at once, each on a stream of its own, so that one
// solve's small kernels and host synchronisations overlap another's H*x.
// The returned occupations put 1 on the blocked orbit (N_Occup, Sec. 4.3).
#include "pd_internal.h"
#include "pairdiag.h"

#include <chrono>
#include <cmath>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

using namespace pd;

namespace {

constexpr int64_t kOddBatchMaxDim = int64_t(1) << 17;   // subspaces this small go through the batch
constexpr int kOddWorkers = 3;                            // host threads for larger subspaces

// e and G on the orbits other than b
void restrict_to(int omega, int b, const double *e, const double *G, double *er, double *Gr)
{
    const int om = omega - 1;
    for (int i = 0, r = 0; i < omega; ++i) {
        if (i == b) continue;
        er[r] = e[i];
        for (int j = 0, c = 0; j < omega; ++j) {
            if (j == b) continue;
            Gr[(size_t)r * om + c] = G[i * omega + j];
            ++c;
        }
        ++r;
    }
}

// One worker's share of the blocked subspaces: its best E_b, vector and
// occupations, on a stream of its own.
struct OddWorker {
    int device = 0;
    cudaStream_t st = nullptr;
    void *v[2] = {nullptr, nullptr};   // v[cur] takes the next solve, v[cur ^ 1] holds the best
    int cur = 0;
    int best = -1;
    double best_e = 0.0;
    pairdiag_info best_info{};
    std::vector<double> best_occ;
    int status = PD_OK;                // PD_OK, PD_ENOCONV, or the first error
    std::string error;
    ~OddWorker()
    {
        if (st) cudaStreamSynchronize(st);
        pool_free(v[0]);
        pool_free(v[1]);
        if (st) cudaStreamDestroy(st);
    }
};

}  // namespace

extern "C" int pairdiag_odd_ground_state(int omega, int n_pairs, const double *e, const double *G, int block,
                                         double tol, const pairdiag_options *opt, pairdiag_mlp_t *mlp,
                                         double *e0, int *block_out, double *energies, double *occ,
                                         double *vec, pairdiag_info *info)
{
    const auto t0 = std::chrono::steady_clock::now();
    if (!e || !G || !e0) return fail(PD_EINVAL, "e, G or e0 is null");
    if (omega < 2 || omega > kMaxOmega) return fail(PD_EINVAL, "omega=%d outside 2..%d", omega, kMaxOmega);
    if (n_pairs < 0 || n_pairs > omega - 1) return fail(PD_EINVAL, "n_pairs=%d outside 0..omega-1", n_pairs);
    if (block < -1 || block >= omega) return fail(PD_EINVAL, "block=%d outside -1..omega-1", block);
    if (!(tol >= 0.0)) return fail(PD_EINVAL, "tol must be >= 0");
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
    if (o.start == PD_START_USER) return fail(PD_EINVAL, "PD_START_USER has no vector per blocked subspace");
    if (o.start == PD_START_MLP && !mlp) return fail(PD_EINVAL, "PD_START_MLP needs a network");

    const int om = omega - 1;
    const int64_t dim = (int64_t)host_binom(om, n_pairs);
    if (energies)
        for (int b = 0; b < omega; ++b) energies[b] = NAN;
    int dev = 0;
    PD_CUDA(cudaGetDevice(&dev));
    int status = PD_OK;
    int best = -1;
    double best_e = 0.0;
    pairdiag_info best_info{};
    std::vector<double> best_occ(om > 0 ? om : 1, 0.0);
    std::vector<int> todo;                      // subspaces solved as handles
    if (block >= 0) todo.push_back(block);
    const bool batched = block < 0 && dim <= kOddBatchMaxDim && o.mode == 0 &&
                         (o.start == PD_START_RANDOM || o.start == PD_START_MLP);
    if (batched) {
        // every subspace in one batched solve
        std::vector<int> oms(omega, om), ns(omega, n_pairs), st_b(omega);
        std::vector<double> e_all((size_t)omega * om), G_all((size_t)omega * om * om), e0_b(omega);
        std::vector<pairdiag_batch_result> res(omega);
        for (int b = 0; b < omega; ++b)
            restrict_to(omega, b, e, G, e_all.data() + (size_t)b * om, G_all.data() + (size_t)b * om * om);
        const int sb = pairdiag_batch_ground_state(omega, oms.data(), ns.data(), e_all.data(), G_all.data(), tol, &o,
                                                   mlp, e0_b.data(), st_b.data(), res.data(), nullptr);
        if (sb != PD_OK && sb != PD_ENOCONV) return sb;
        if (sb == PD_ENOCONV) status = PD_ENOCONV;
        for (int b = 0; b < omega; ++b) {
            const double eb = e0_b[b] + e[b];
            if (energies) energies[b] = eb;
            if (best < 0 || eb < best_e) {
                best = b;
                best_e = eb;
            }
        }
        const pairdiag_batch_result &rb = res[best];
        best_info.dim = dim;
        best_info.nnz_offdiag = dim * (int64_t)n_pairs * (int64_t)(om - n_pairs);
        best_info.iterations = rb.iterations;
        best_info.hx_products = rb.iterations;
        best_info.converged = rb.converged;
        best_info.rel_residual = rb.rel_residual;
        best_info.gap_estimate = NAN;
        if (vec || occ) todo.push_back(best);   // the winner once more, for its vector
    } else if (block < 0) {
        for (int b = 0; b < omega; ++b) todo.push_back(b);
    }

    // per-subspace start weights of the learned start, computed here: the
    // network serves one call at a time, the workers solve concurrently
    std::vector<std::vector<double>> wts(omega);
    if (o.start == PD_START_MLP && mlp)
        for (int b : todo) {
            std::vector<double> er(om), Gr((size_t)om * om);
            restrict_to(omega, b, e, G, er.data(), Gr.data());
            wts[b].assign(om, 0.0);
            PD_TRY(mlp_predict(mlp, om, n_pairs, er.data(), Gr.data(), wts[b].data()));
        }

    const int nwork = std::max(1, std::min<int>(kOddWorkers, (int)todo.size()));
    std::vector<OddWorker> work(nwork);
    auto run = [&](int wi) {
        OddWorker &W = work[wi];
        auto bad = [&](int code) {
            if (W.status == PD_OK || W.status == PD_ENOCONV) {
                W.status = code;
                W.error = pairdiag_last_error();
            }
        };
        if (cudaSetDevice(dev) != cudaSuccess) { bad(fail(PD_ECUDA, "odd: cudaSetDevice")); return; }
        if (cudaStreamCreateWithFlags(&W.st, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            bad(fail(PD_ECUDA, "odd: stream creation failed"));
            return;
        }
        for (int k = 0; k < 2; ++k) {
            const cudaError_t ce = pool_alloc(&W.v[k], sizeof(double) * (size_t)dim);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                bad(fail(ce == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA, "odd: %s", cudaGetErrorString(ce)));
                return;
            }
        }
        W.best_occ.assign(om > 0 ? om : 1, 0.0);
        std::vector<double> er(om), Gr((size_t)om * om);
        for (size_t t = wi; t < todo.size(); t += nwork) {
            const int b = todo[t];
            restrict_to(omega, b, e, G, er.data(), Gr.data());
            pairdiag_t *h = nullptr;
            int st = pairdiag_create(om, n_pairs, er.data(), Gr.data(), &o, &h);
            if (st != PD_OK) { bad(st); return; }
            st = pairdiag_set_stream(h, W.st);
            if (st == PD_OK && !wts[b].empty()) st = pairdiag_set_start_weights(h, wts[b].data());
            double eb = 0.0;
            pairdiag_info ib{};
            if (st == PD_OK) st = pairdiag_ground_state_dev(h, tol, &eb, static_cast<double *>(W.v[W.cur]), &ib);
            if (st != PD_OK && st != PD_ENOCONV) {
                pairdiag_destroy(h);
                bad(st);
                return;
            }
            if (st == PD_ENOCONV && W.status == PD_OK) W.status = PD_ENOCONV;
            eb += e[b];
            if (batched) eb = best_e;               // E_b stays the batched solve's (the vector is this solve's)
            if (energies) energies[b] = eb;         // distinct b per worker
            if (W.best < 0 || eb < W.best_e) {
                if (occ) {
                    const int so = pairdiag_occupations_dev(h, static_cast<const double *>(W.v[W.cur]),
                                                            W.best_occ.data());
                    if (so != PD_OK) {
                        pairdiag_destroy(h);
                        bad(so);
                        return;
                    }
                }
                W.best = b;
                W.best_e = eb;
                W.best_info = ib;
                W.cur ^= 1;
            }
            pairdiag_destroy(h);
        }
    };
    if (!todo.empty()) {
        if (nwork == 1) {
            run(0);
        } else {
            std::vector<std::thread> th;
            for (int wi = 0; wi < nwork; ++wi) th.emplace_back(run, wi);
            for (auto &t : th) t.join();
        }
    }
    // the first error of any worker, then the lowest E_b over the workers
    for (const OddWorker &W : work)
        if (W.status != PD_OK && W.status != PD_ENOCONV) return fail(W.status, "%s", W.error.c_str());
    const OddWorker *win = nullptr;
    for (const OddWorker &W : work) {
        if (W.status == PD_ENOCONV) status = PD_ENOCONV;
        if (W.best >= 0 && (!win || W.best_e < win->best_e)) win = &W;
    }
    if (win) {
        best = win->best;
        best_e = win->best_e;
        best_info = win->best_info;
        best_occ = win->best_occ;
    }
    if (vec) {
        if (!win) return fail(PD_ECUDA, "odd: no vector computed");
        PD_CUDA(cudaMemcpy(vec, win->v[win->cur ^ 1], sizeof(double) * (size_t)dim, cudaMemcpyDeviceToHost));
    }
    if (occ)
        for (int i = 0, r = 0; i < omega; ++i) occ[i] = (i == best) ? 1.0 : best_occ[r++];
    *e0 = best_e;
    if (block_out) *block_out = best;
    if (info) {
        *info = best_info;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status == PD_ENOCONV) return fail(PD_ENOCONV, "odd: a blocked subspace missed tol %.3g", tol);
    return PD_OK;
}
