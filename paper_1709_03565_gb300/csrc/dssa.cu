// Influence maximisation with DSSA-style doubling over SKIS sketches (Sec. V-B;
// the DSSA stop rule with SKIS samples in the appendix, "Improvements of
// SSA/DSSA using SKIS sketch").
//
// Two independent sketches R and R^c (own Philox keys) start at n0 samples
// and double in place, round t = 1, 2, ...: greedy (Alg. 3) on R gives S_k;
// S_k is re-estimated on R^c; the run stops when Cov_R(S_k) >= Lambda_2 and
//   (e1 + e2 + e1 e2)(1 - 1/e - eps) + (1 - 1/e) e3 <= eps,
//   e1 = I_R / I_Rc - 1,
//   e2 = eps sqrt(n (1 + eps) / (2^(t-1) I_Rc)),
//   e3 = eps sqrt(n (1 + eps)(1 - 1/e - eps) / ((1 + eps/3) 2^(t-1) I_Rc)),
// or when the samples reach n_max. Estimates are formed on the host from the
// exact integers (coverage, W, T, sum of 2^f - w_v) with correctly rounded
// conversions, in the order written here, so the decisions are reproducible.
#include <cmath>
#include <string>
#include <vector>

#include "../../include/skis.h"
#include "skis_internal.cuh"

using namespace skis;

namespace {

constexpr double kInvE = 0.36787944117144233;  // e^-1 rounded to binary64

__global__ void k_gather_w(const uint64_t* __restrict__ w, const int32_t* __restrict__ idx, int32_t k,
                           uint64_t* __restrict__ out) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) out[i] = w[idx[i]];
}

double exact_estimate(uint64_t cov, uint64_t W, uint64_t T, u128 sum_c, int f) {
    const u128 N = (u128)cov * W + (u128)T * sum_c;
    const u128 D = (u128)T << f;
    return (double)N / (double)D;  // both conversions correctly rounded
}

}  // namespace

extern "C" int skis_dssa_maxinf(const skis_graph* g, uint64_t seed_r, uint64_t seed_rc, int32_t k, double eps,
                                double delta, uint64_t lambda2, uint64_t n0, uint64_t n_max, int32_t* seeds_out,
                                skis_dssa_result* res, void* cuda_stream) {
    if (!g || !seeds_out || !res) return set_last_error(SKIS_EINVAL, "skis_dssa_maxinf: NULL argument");
    if (k < 1 || k > g->n) return set_last_error(SKIS_EINVAL, "skis_dssa_maxinf: k must be in [1, n]");
    if (!(eps > 0.0 && eps < 1.0 - kInvE)) return set_last_error(SKIS_EINVAL, "skis_dssa_maxinf: eps must be in (0, 1 - 1/e)");
    if (!(delta > 0.0 && delta < 1.0)) return set_last_error(SKIS_EINVAL, "skis_dssa_maxinf: delta must be in (0, 1)");
    if (n0 < 1 || n_max < n0 || n_max >= (1ull << 32))
        return set_last_error(SKIS_EINVAL, "skis_dssa_maxinf: need 1 <= n0 <= n_max < 2^32");
    if (g->W == 0) return set_last_error(SKIS_EINVAL, "skis_dssa_maxinf: Gamma = 0");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const double n = (double)g->n;
    const double gamma_n = ((double)g->W / (double)(1ull << g->f)) / n;
    int t_max = 1;
    for (uint64_t N = n0; N < n_max; N *= 2) ++t_max;
    if (lambda2 == 0) {
        // reading of Lambda_2 = O(Gamma/n log(t_max/delta) eps^-2): the constant of
        // Lemma 7's (eps, delta) sample count, (2 Gamma/n + 2 eps/3) ln(2 t_max / delta) / eps^2
        const double l = (2.0 * gamma_n + 2.0 * eps / 3.0) * std::log(2.0 * (double)t_max / delta) / (eps * eps);
        lambda2 = (uint64_t)std::ceil(l);
    }
    skis_sketch R, Rc;
    R.g = g;
    R.seed = seed_r;
    R.stream = st;
    Rc.g = g;
    Rc.seed = seed_rc;
    Rc.stream = st;
    std::string err;
    int rc = SKIS_OK;
    std::vector<int64_t> cov(k);
    std::vector<double> est(k);
    std::vector<uint64_t> wsel(k);
    int32_t* d_sel = nullptr;
    uint64_t* d_w = nullptr;
    int64_t* d_q = nullptr;
    int64_t* d_cov = nullptr;
    double* d_est = nullptr;
    auto cuda = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == SKIS_OK) {
            rc = e == cudaErrorMemoryAllocation ? SKIS_ENOMEM : SKIS_ERR_CUDA;
            err = std::string("CUDA error: ") + cudaGetErrorString(e);
        }
        return rc == SKIS_OK;
    };
    cuda(dev_alloc_t(&d_sel, (size_t)k, st));
    cuda(dev_alloc_t(&d_w, (size_t)k, st));
    cuda(dev_alloc_t(&d_q, 2, st));
    cuda(dev_alloc_t(&d_cov, 1, st));
    cuda(dev_alloc_t(&d_est, 1, st));
    uint64_t N = n0;
    int t = 1;
    skis_dssa_result out{};
    out.lambda2 = lambda2;
    while (rc == SKIS_OK) {
        // grow both sketches in place to N samples
        rc = sketch_sample(&R, N - R.T, st, &err);
        if (rc == SKIS_OK) rc = sketch_sample(&Rc, N - Rc.T, st, &err);
        if (rc != SKIS_OK) break;
        rc = sketch_greedy(&R, k, seeds_out, cov.data(), est.data(), st, &err);
        if (rc != SKIS_OK) break;
        // sum over S_k of 2^f - w_v, exactly
        if (!cuda(cudaMemcpyAsync(d_sel, seeds_out, (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, st))) break;
        k_gather_w<<<(k + 255) / 256, 256, 0, st>>>(g->w, d_sel, k, d_w); note_launch();
        if (!cuda(cudaGetLastError())) break;
        if (!cuda(cudaMemcpyAsync(wsel.data(), d_w, (size_t)k * sizeof(uint64_t), cudaMemcpyDeviceToHost, st))) break;
        if (!cuda(cudaStreamSynchronize(st))) break;
        u128 sum_c = 0;
        for (int32_t i = 0; i < k; ++i) sum_c += (u128)((1ull << g->f) - wsel[i]);
        // Cov_{R^c}(S_k)
        const int64_t h_q[2] = {0, k};
        if (!cuda(cudaMemcpyAsync(d_q, h_q, sizeof(h_q), cudaMemcpyHostToDevice, st))) break;
        rc = sketch_estimate(&Rc, 1, d_q, d_sel, h_q, d_cov, d_est, st, &err);
        if (rc != SKIS_OK) break;
        int64_t cov_c = 0;
        if (!cuda(cudaMemcpyAsync(&cov_c, d_cov, sizeof(int64_t), cudaMemcpyDeviceToHost, st))) break;
        if (!cuda(cudaStreamSynchronize(st))) break;
        const uint64_t cov_r = (uint64_t)cov[k - 1];
        const double i_r = exact_estimate(cov_r, g->W, N, sum_c, g->f);
        const double i_c = exact_estimate((uint64_t)cov_c, g->W, N, sum_c, g->f);
        const double scale = std::ldexp(1.0, t - 1);  // 2^(t-1)
        const double e1 = i_r / i_c - 1.0;
        const double e2 = eps * std::sqrt(n * (1.0 + eps) / (scale * i_c));
        const double e3 = eps * std::sqrt(n * (1.0 + eps) * (1.0 - kInvE - eps) / ((1.0 + eps / 3.0) * scale * i_c));
        out.rounds = t;
        out.samples = N;
        out.coverage = (int64_t)cov_r;
        out.coverage_c = cov_c;
        out.estimate = i_r;
        out.estimate_c = i_c;
        out.eps1 = e1;
        out.eps2 = e2;
        out.eps3 = e3;
        if (cov_r >= lambda2) {
            const double lhs = (e1 + e2 + e1 * e2) * (1.0 - kInvE - eps) + (1.0 - kInvE) * e3;
            if (lhs <= eps) {
                out.stopped_by = 1;
                break;
            }
        }
        if (N >= n_max) {
            out.stopped_by = 2;
            break;
        }
        N = std::min<uint64_t>(N * 2, n_max);
        ++t;
    }
    sketch_release(&R);
    sketch_release(&Rc);
    dev_free(d_sel, st);
    dev_free(d_w, st);
    dev_free(d_q, st);
    dev_free(d_cov, st);
    dev_free(d_est, st);
    if (rc != SKIS_OK) return set_last_error(rc, "skis_dssa_maxinf: " + err);
    *res = out;
    return SKIS_OK;
}
