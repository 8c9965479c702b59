// pd_odd.cu -- odd-mass systems in the blocking approximation (Eq. 3).
//
// One unpaired particle in orbit b keeps every pair out of b, so the
// seniority-one subspace with b blocked is the seniority-zero space of the
// pairs on the other Omega-1 orbits, and H_b there is the constant e_b plus
// Eq. 2 restricted to those orbits.  Each subspace is therefore an ordinary
// handle of this library on the reduced (e, G): the same basis tables, H*x
// kernels and Lanczos run unchanged.  Block = 0 of the paper (block = -1
// here) needs every b: the Omega subspaces, all of the same size, are solved
// together by the batched solver (pd_batch.cu) and the lowest E_b is kept;
// when the caller wants its vector or occupations, that one subspace is
// solved once more as a handle.  Start kinds the batch does not offer (the
// paper's [1,0,...,0] and HF) solve the subspaces one after another.  The
// returned occupations put 1 on the blocked orbit (N_Occup, Sec. 4.3).
#include "pd_internal.h"
#include "pairdiag.h"

#include <chrono>
#include <cmath>
#include <utility>
#include <vector>

using namespace pd;

namespace {

struct OddBuffers {
    void *v[2] = {nullptr, nullptr};
    ~OddBuffers()
    {
        if (v[0] || v[1]) cudaDeviceSynchronize();
        pool_free(v[0]);
        pool_free(v[1]);
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
    OddBuffers buf;
    for (int k = 0; k < 2; ++k) {
        const cudaError_t ce = pool_alloc(&buf.v[k], sizeof(double) * (size_t)dim);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return fail(ce == cudaErrorMemoryAllocation ? PD_ENOMEM : PD_ECUDA, "odd: %s", cudaGetErrorString(ce));
        }
    }
    int cur = 0;                              // buf.v[cur] takes the next solve, buf.v[cur ^ 1] holds the best
    int best = -1;
    double best_e = 0.0;
    pairdiag_info best_info{};
    std::vector<double> best_occ(om > 0 ? om : 1, 0.0);
    std::vector<double> er(om);
    std::vector<double> Gr((size_t)om * om);
    int status = PD_OK;
    int b_lo = block < 0 ? 0 : block, b_hi = block < 0 ? omega - 1 : block;
    const bool batched = block < 0 && o.mode == 0 && (o.start == PD_START_RANDOM || o.start == PD_START_MLP);
    if (batched) {
        // every subspace in one batched solve
        std::vector<int> oms(omega, om), ns(omega, n_pairs), st_b(omega);
        std::vector<double> e_all((size_t)omega * om), G_all((size_t)omega * om * om), e0_b(omega);
        std::vector<pairdiag_batch_result> res(omega);
        for (int b = 0; b < omega; ++b)
            for (int i = 0, r = 0; i < omega; ++i) {
                if (i == b) continue;
                e_all[(size_t)b * om + r] = e[i];
                for (int j = 0, c = 0; j < omega; ++j) {
                    if (j == b) continue;
                    G_all[((size_t)b * om + r) * om + c] = G[i * omega + j];
                    ++c;
                }
                ++r;
            }
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
        if (!vec && !occ) b_hi = b_lo - 1;         // nothing more to compute
        else b_lo = b_hi = best;                    // the winner once more, for its vector
    }
    for (int b = b_lo; b <= b_hi; ++b) {
        for (int i = 0, r = 0; i < omega; ++i) {          // e and G on the orbits other than b
            if (i == b) continue;
            er[r] = e[i];
            for (int j = 0, c = 0; j < omega; ++j) {
                if (j == b) continue;
                Gr[(size_t)r * om + c] = G[i * omega + j];
                ++c;
            }
            ++r;
        }
        pairdiag_t *h = nullptr;
        PD_TRY(pairdiag_create(om, n_pairs, er.data(), Gr.data(), &o, &h));
        int st = PD_OK;
        if (mlp) st = pairdiag_set_mlp(h, mlp);
        double eb = 0.0;
        pairdiag_info ib{};
        if (st == PD_OK) st = pairdiag_ground_state_dev(h, tol, &eb, static_cast<double *>(buf.v[cur]), &ib);
        if (st != PD_OK && st != PD_ENOCONV) {
            pairdiag_destroy(h);
            return st;
        }
        if (st == PD_ENOCONV) status = PD_ENOCONV;
        eb += e[b];
        if (batched) eb = best_e;                  // E_b stays the batched solve's (the vector is this solve's)
        if (energies) energies[b] = eb;
        if (batched || best < 0 || eb < best_e) {
            if (occ) {
                const int so = pairdiag_occupations_dev(h, static_cast<const double *>(buf.v[cur]), best_occ.data());
                if (so != PD_OK) {
                    pairdiag_destroy(h);
                    return so;
                }
            }
            best = b;
            best_e = eb;
            best_info = ib;
            cur ^= 1;
        }
        pairdiag_destroy(h);
    }
    const void *vbest = buf.v[cur ^ 1];
    if (vec) PD_CUDA(cudaMemcpy(vec, vbest, sizeof(double) * (size_t)dim, cudaMemcpyDeviceToHost));
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
