// hd_tune.cu -- candidate enumeration, device-timed autotuning and the
// process-wide tuning cache (the paper's empirical optimizer, Section 7:
// scan the FFT size m and the residue blocking, time, keep the fastest).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "hd_plan.h"

namespace hd {

namespace {

bool desc_ok_1d(const hd_desc* d) {
    if (!d || d->ndim != 1) return false;
    if (d->kind < HD_COMPLEX || d->kind > HD_HERMITIAN) return false;
    if (d->dtype != HD_F32 && d->dtype != HD_F64) return false;
    if (!mult_counts_ok(d->mult, d->A, d->B)) return false;
    return d->L[0] > 0 && d->M[0] > 0;
}

// (p, q) pairs worth trying for one m: the paper's derivation, and for p > 2
// the explicit padding to the next power-of-two p (p m >= L holds for both).
void pq_options(int kind, int64_t L, int64_t M, int64_t m, std::vector<std::pair<int64_t, int64_t>>* out) {
    int64_t p, q, n;
    hd_derive_params(kind, L, M, m, &p, &q, &n);
    out->push_back({p, q});
    if (kind == HD_COMPLEX && p > 2 && !is_pow2(p)) {
        int64_t pp = next_pow2_t(p);
        out->push_back({pp, ceil_div(M, pp * m) * pp});
    }
    if (kind != HD_COMPLEX && p > 2 && !is_pow2(p / 2)) {
        int64_t pp = 2 * next_pow2_t(p / 2);
        out->push_back({pp, ceil_div(2 * M, pp * m) * (pp / 2)});
    }
}

}  // namespace

int enumerate_candidates(const hd_desc* d, std::vector<hd_candidate>* out) {
    out->clear();
    const int64_t L = d->L[0], M = d->M[0];
    if (M < hd_dealias_bound(d->kind, d->mult, L)) return 0;
    std::vector<std::tuple<int64_t, int64_t, int64_t>> mpq;
    for (int64_t m = 1; m <= 8192; m <<= 1) {
        std::vector<std::pair<int64_t, int64_t>> opts;
        pq_options(d->kind, L, M, m, &opts);
        for (auto& o : opts) mpq.emplace_back(m, o.first, o.second);
    }
    mpq.emplace_back(next_pow2_t(M), 1, 1);   // explicit zero padding
    Conv1dCfg vars[64];
    const int nv = conv1d_variants(d->dtype, d->kind, vars, 64);
    for (auto& t : mpq) {
        int64_t m = std::get<0>(t), p = std::get<1>(t), q = std::get<2>(t), S, n;
        int nb;
        if (validate_axis(d->kind, d->mult, L, M, m, p, q, &S, &n, &nb) != HD_OK) continue;
        const bool comp = d->dtype == HD_F32 && comp_default(n);
        const int64_t Ls = d->kind == HD_HERMITIAN ? (L + 1) / 2 : L;
        if (split_supported(d->dtype, d->kind, d->mult, S, nb)) {
            bool dup = false;
            for (auto& c : *out)
                if (c.S == S && c.n == n) {
                    if (p < c.p) {
                        c.m = m;
                        c.p = p;
                        c.q = q;
                    }
                    dup = true;
                }
            if (!dup) {
                hd_candidate c;
                std::memset(&c, 0, sizeof(c));
                c.m = m;
                c.p = p;
                c.q = q;
                c.D = 1;
                c.S = S;
                c.n = n;
                c.E = 8;
                c.minb = 1;
                c.comp = comp ? 1 : 0;
                out->push_back(c);
            }
            continue;
        }
        for (int v = 0; v < nv && v < 64; ++v) {
            if (vars[v].S != S) continue;
            if (!fused_supported(d->dtype, d->kind, d->mult, S, nb, Ls, comp, vars[v].E, vars[v].minb)) continue;
            // identical kernel work (same S, n, variant): keep the smallest p
            bool dup = false;
            for (auto& c : *out) {
                if (c.S == S && c.n == n && c.E == vars[v].E && c.minb == vars[v].minb && single_group(d->kind, c)) {
                    if (p < c.p) {
                        c.m = m;
                        c.p = p;
                        c.q = q;
                    }
                    dup = true;
                    break;
                }
            }
            if (dup) continue;
            hd_candidate c;
            std::memset(&c, 0, sizeof(c));
            c.m = m;
            c.p = p;
            c.q = q;
            c.D = d->kind == HD_HERMITIAN ? 2 : 1;
            c.S = S;
            c.n = n;
            c.E = vars[v].E;
            c.minb = vars[v].minb;
            c.comp = comp ? 1 : 0;
            c.ms = 0;
            out->push_back(c);
        }
        // D > 1 residues per pass (Section 6.5) for few convolutions: D residue
        // groups of one convolution run at once on a thread-block cluster
        if (d->kind != HD_HERMITIAN && !split_supported(d->dtype, d->kind, d->mult, S, nb)) {
            for (int ci = 0; ci < 6; ++ci) {
                const int D = ci < 3 ? 2 : 4, E = 8 >> (ci % 3);
                if (D > n || !cluster_supported(d->dtype, d->kind, d->mult, S, nb, Ls, D, E)) continue;
                bool dup = false;
                for (auto& c : *out) {
                    if (c.S == S && c.n == n && c.D == D && c.E == E) {
                        if (p < c.p) {
                            c.m = m;
                            c.p = p;
                            c.q = q;
                        }
                        dup = true;
                        break;
                    }
                }
                if (dup) continue;
                hd_candidate c;
                std::memset(&c, 0, sizeof(c));
                c.m = m;
                c.p = p;
                c.q = q;
                c.D = D;
                c.S = S;
                c.n = n;
                c.E = E;
                c.minb = 1;
                c.comp = 0;
                out->push_back(c);
            }
        }
    }
    return (int)out->size();
}

namespace {

struct CacheKey {
    int dtype, kind, mult;
    int64_t L, M;
    bool operator<(const CacheKey& o) const {
        return std::tie(dtype, kind, mult, L, M) < std::tie(o.dtype, o.kind, o.mult, o.L, o.M);
    }
};
std::mutex g_cache_mu;
std::map<CacheKey, hd_candidate>& cache() {
    static std::map<CacheKey, hd_candidate> c;
    return c;
}
CacheKey key_of(const hd_desc* d) { return CacheKey{d->dtype, d->kind, d->mult, d->L[0], d->M[0]}; }

// better(a, b): a is faster beyond 1%, or within 1% with smaller q m, then smaller m
bool better(const hd_candidate& a, const hd_candidate& b) {
    if (a.ms < b.ms * 0.99) return true;
    if (a.ms > b.ms * 1.01) return false;
    const int64_t qa = a.n * a.S, qb = b.n * b.S;
    if (qa != qb) return qa < qb;
    if (a.m != b.m) return a.m < b.m;
    return a.ms < b.ms;
}

}  // namespace

bool cache_lookup(const hd_desc* d, hd_candidate* c) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    auto it = cache().find(key_of(d));
    if (it == cache().end()) return false;
    *c = it->second;
    return true;
}

// Timed search used when the selector is unsure: the batch size gives about
// 2^21 stored values per timed call.
hd_status timed_choice(const hd_desc* d, bool (*ok)(const hd_desc*, const hd_candidate&), hd_candidate* out) {
    int64_t count = ((int64_t)1 << 21) / std::max<int64_t>(d->L[0], 64);
    count = std::max<int64_t>(1, std::min<int64_t>(count, 4096));
    std::vector<hd_candidate> all(256);
    int n = 0;
    hd_candidate best;
    hd_status st = hd_autotune(d, count, 3, all.data(), (int)all.size(), &n, &best);
    if (st != HD_OK) return st;
    bool found = false;
    for (int i = 0; i < n && i < (int)all.size(); ++i) {
        if (all[i].ms <= 0 || (ok && !ok(d, all[i]))) continue;
        if (!found || all[i].ms < out->ms) {
            *out = all[i];
            found = true;
        }
    }
    return found ? HD_OK : HD_ERR_UNSUPPORTED;
}

}  // namespace hd

using namespace hd;

extern "C" {

hd_status hd_enumerate_candidates(const hd_desc* d, hd_candidate* out, int cap, int* count) {
    if (!desc_ok_1d(d) || !count || cap < 0 || (cap > 0 && !out)) return HD_ERR_INVALID;
    std::vector<hd_candidate> v;
    enumerate_candidates(d, &v);
    for (int i = 0; i < (int)v.size() && i < cap; ++i) out[i] = v[i];
    *count = (int)v.size();
    return HD_OK;
}

hd_status hd_plan_create_candidate(hd_plan** out, const hd_desc* d, const hd_candidate* c) {
    if (!out || !d || !c) return HD_ERR_INVALID;
    *out = nullptr;
    if (!desc_ok_1d(d)) return HD_ERR_INVALID;
    return plan_create_from(out, d, c);
}

hd_status hd_autotune(const hd_desc* d, int64_t count, int reps, hd_candidate* outc, int cap, int* nout,
                      hd_candidate* best) {
    if (!desc_ok_1d(d) || count <= 0 || reps <= 0 || cap < 0 || (cap > 0 && !outc)) return HD_ERR_INVALID;
    std::vector<hd_candidate> cands;
    enumerate_candidates(d, &cands);
    if (cands.empty()) return HD_ERR_UNSUPPORTED;
    const int64_t Ls = d->kind == HD_HERMITIAN ? (d->L[0] + 1) / 2 : d->L[0];
    const size_t esz = d->dtype == HD_F64 ? 16 : 8;
    const size_t bytes = (size_t)count * (size_t)Ls * esz;
    constexpr int kBufs = kMaxIn + kMaxOut;
    void* buf[kBufs] = {};
    hd_status st = HD_OK;
    if (d->A + d->B > kBufs) return HD_ERR_INVALID;
    for (int a = 0; a < d->A + d->B && st == HD_OK; ++a) {   // A inputs, B outputs
        if (cudaMalloc(&buf[a], bytes) != cudaSuccess) st = HD_ERR_NOMEM;
        else if (cudaMemset(buf[a], 0, bytes) != cudaSuccess) st = HD_ERR_CUDA;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == HD_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = HD_ERR_CUDA;
    std::vector<float> t;
    for (size_t i = 0; i < cands.size() && st == HD_OK; ++i) {
        hd_plan* pl = nullptr;
        hd_status ps = plan_create_from(&pl, d, &cands[i]);
        if (ps != HD_OK) {
            cands[i].ms = -1;
            continue;
        }
        const void* f[kMaxIn];
        for (int a = 0; a < kMaxIn; ++a) f[a] = buf[a];
        void* h[kMaxOut] = {};
        for (int b = 0; b < d->B && b < kMaxOut; ++b) h[b] = buf[d->A + b];
        t.clear();
        for (int r = 0; r < 2 + reps && st == HD_OK; ++r) {
            cudaEventRecord(e0, 0);
            if (plan_execute(pl, count, f, h, Ls, 0) != HD_OK) st = HD_ERR_CUDA;
            cudaEventRecord(e1, 0);
            if (cudaEventSynchronize(e1) != cudaSuccess) st = HD_ERR_CUDA;
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            if (r >= 2) t.push_back(ms);
        }
        std::sort(t.begin(), t.end());
        cands[i].ms = t.empty() ? -1 : t[t.size() / 2];
        plan_free(pl);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    for (int a = 0; a < kBufs; ++a)
        if (buf[a]) cudaFree(buf[a]);
    if (st != HD_OK) {
        cudaGetLastError();
        return st;
    }
    int bi = -1;
    for (size_t i = 0; i < cands.size(); ++i) {
        if (cands[i].ms <= 0) continue;
        if (bi < 0 || better(cands[i], cands[bi])) bi = (int)i;
    }
    if (bi < 0) return HD_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> g(g_cache_mu);
        cache()[key_of(d)] = cands[bi];
    }
    for (int i = 0; i < (int)cands.size() && i < cap; ++i) outc[i] = cands[i];
    if (nout) *nout = (int)cands.size();
    if (best) *best = cands[bi];
    return HD_OK;
}

hd_status hd_tune_cache_put(const hd_desc* d, const hd_candidate* c) {
    if (!desc_ok_1d(d) || !c) return HD_ERR_INVALID;
    std::lock_guard<std::mutex> g(g_cache_mu);
    cache()[key_of(d)] = *c;
    return HD_OK;
}

hd_status hd_tune_cache_get(const hd_desc* d, hd_candidate* c) {
    if (!desc_ok_1d(d) || !c) return HD_ERR_INVALID;
    return cache_lookup(d, c) ? HD_OK : HD_ERR_INVALID;
}

hd_status hd_tune_cache_clear(void) {
    std::lock_guard<std::mutex> g(g_cache_mu);
    cache().clear();
    return HD_OK;
}

}  // extern "C"
