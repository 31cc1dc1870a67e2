// hd_selector.cu -- candidate selection by an installed ensemble of MLPs
// (hd_mlp.cu) that predict the log time of one convolution for a (problem,
// candidate) pair; the timed search (hd_autotune) is the fallback when the
// ensemble is unsure.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "hd_plan.h"

namespace hd {

namespace {

std::mutex g_sel_mu;
std::vector<hd_mlp*> g_models;
float g_tau = 0.05f, g_sigma = 0.25f;
int g_fallback = 1;

}  // namespace

void selector_features(const hd_desc* d, const hd_candidate* c, float* f) {
    const double L = (double)d->L[0], M = (double)d->M[0];
    f[0] = (float)(std::log2(L) / 16.0);
    f[1] = (float)(std::log2(M) / 16.0);
    f[2] = (float)(L / M);
    f[3] = (float)(d->A - 2);
    f[4] = d->kind == HD_CENTERED ? 1.0f : 0.0f;
    f[5] = d->kind == HD_HERMITIAN ? 1.0f : 0.0f;
    f[6] = d->dtype == HD_F64 ? 1.0f : 0.0f;
    f[7] = (float)(std::log2((double)c->S) / 16.0);
    f[8] = (float)(std::log2((double)c->n) / 8.0);
    f[9] = (float)(((double)c->n * (double)c->S - M) / M);
    f[10] = c->S > max_fused_S(d->dtype) ? 1.0f : 0.0f;
    f[11] = (float)c->E / 16.0f;
    f[12] = (float)(c->minb - 1);
}

bool selector_installed() {
    std::lock_guard<std::mutex> g(g_sel_mu);
    return !g_models.empty();
}

// For each problem i with candidate list cands[i] (non-empty), picks pick[i]
// (index into cands[i]) and reports whether the ensemble was confident.
hd_status selector_choose_batch(const std::vector<const hd_desc*>& descs,
                                const std::vector<std::vector<hd_candidate>>& cands, std::vector<int>* pick,
                                std::vector<int>* confident) {
    std::lock_guard<std::mutex> g(g_sel_mu);
    if (g_models.empty()) return HD_ERR_INVALID;
    const int NF = HD_SELECTOR_FEATURES;
    std::vector<float> X;
    std::vector<int64_t> start(descs.size() + 1, 0);
    for (size_t i = 0; i < descs.size(); ++i) {
        start[i + 1] = start[i] + (int64_t)cands[i].size();
        for (auto& c : cands[i]) {
            float f[HD_SELECTOR_FEATURES];
            selector_features(descs[i], &c, f);
            X.insert(X.end(), f, f + NF);
        }
    }
    const int64_t N = start.back();
    pick->assign(descs.size(), 0);
    confident->assign(descs.size(), 0);
    if (N == 0) return HD_OK;
    float *dX = nullptr, *dY = nullptr;
    if (cudaMalloc(&dX, sizeof(float) * X.size()) != cudaSuccess || cudaMalloc(&dY, sizeof(float) * N) != cudaSuccess) {
        cudaFree(dX);
        cudaGetLastError();
        return HD_ERR_NOMEM;
    }
    std::vector<std::vector<float>> Y(g_models.size(), std::vector<float>(N));
    hd_status st = cudaMemcpy(dX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice) == cudaSuccess ? HD_OK
                                                                                                         : HD_ERR_CUDA;
    for (size_t k = 0; k < g_models.size() && st == HD_OK; ++k) {
        st = hd_mlp_forward(g_models[k], dX, N, dY, nullptr);
        if (st == HD_OK && cudaMemcpy(Y[k].data(), dY, sizeof(float) * N, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = HD_ERR_CUDA;
    }
    cudaFree(dX);
    cudaFree(dY);
    if (st != HD_OK) {
        cudaGetLastError();
        return st;
    }
    const size_t K = g_models.size();
    for (size_t i = 0; i < descs.size(); ++i) {
        int best = -1, second = -1;
        double mb = 0, m2 = 0, sb = 0;
        std::vector<int> votes(cands[i].size(), 0);
        for (size_t k = 0; k < K; ++k) {
            int kb = 0;
            for (int64_t j = start[i]; j < start[i + 1]; ++j)
                if (Y[k][j] < Y[k][start[i] + kb]) kb = (int)(j - start[i]);
            votes[kb]++;
        }
        for (int64_t j = start[i]; j < start[i + 1]; ++j) {
            double mu = 0, s2 = 0;
            for (size_t k = 0; k < K; ++k) mu += Y[k][j];
            mu /= (double)K;
            for (size_t k = 0; k < K; ++k) s2 += (Y[k][j] - mu) * (Y[k][j] - mu);
            const double sd = K > 1 ? std::sqrt(s2 / (double)(K - 1)) : 0.0;
            const int jj = (int)(j - start[i]);
            if (best < 0 || mu < mb) {
                second = best;
                m2 = mb;
                best = jj;
                mb = mu;
                sb = sd;
            } else if (second < 0 || mu < m2) {
                second = jj;
                m2 = mu;
            }
        }
        (*pick)[i] = best;
        const bool agree = votes[best] == (int)K;
        const bool spread_ok = sb <= g_sigma;
        const bool margin_ok = second < 0 || (m2 - mb) >= g_tau;
        (*confident)[i] = (spread_ok && (agree || margin_ok)) ? 1 : 0;
    }
    return HD_OK;
}

int selector_fallback() {
    std::lock_guard<std::mutex> g(g_sel_mu);
    return g_fallback;
}

}  // namespace hd

using namespace hd;

extern "C" {

hd_status hd_selector_features(const hd_desc* d, const hd_candidate* c, float* out) {
    if (!d || !c || !out || d->L[0] <= 0 || d->M[0] <= 0 || c->S <= 0 || c->n <= 0) return HD_ERR_INVALID;
    selector_features(d, c, out);
    return HD_OK;
}

hd_status hd_selector_install(hd_mlp* const* models, int k, float tau, float sigma, int fallback) {
    if (!models || k <= 0 || k > 64 || !(tau >= 0) || !(sigma >= 0)) return HD_ERR_INVALID;
    for (int i = 0; i < k; ++i)
        if (!models[i] || hd_mlp_num_params(models[i]) <= 0) return HD_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_sel_mu);
    g_models.assign(models, models + k);
    g_tau = tau;
    g_sigma = sigma;
    g_fallback = fallback ? 1 : 0;
    return HD_OK;
}

hd_status hd_selector_clear(void) {
    std::lock_guard<std::mutex> g(g_sel_mu);
    g_models.clear();
    return HD_OK;
}

hd_status hd_selector_choose(const hd_desc* d, hd_candidate* out, int* confident) {
    if (!d || !out || d->ndim != 1) return HD_ERR_INVALID;
    std::vector<hd_candidate> all, c;
    enumerate_candidates(d, &all);
    for (auto& x : all)
        if (single_group(d->kind, x)) c.push_back(x);
    if (c.empty()) return HD_ERR_UNSUPPORTED;
    std::vector<int> pick, conf;
    hd_status st = selector_choose_batch({d}, {c}, &pick, &conf);
    if (st != HD_OK) return st;
    *out = c[pick[0]];
    if (confident) *confident = conf[0];
    return HD_OK;
}

}  // extern "C"
