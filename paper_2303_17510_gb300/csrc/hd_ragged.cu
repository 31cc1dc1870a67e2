// hd_ragged.cu -- ragged batches in one persistent launch (see hd_ragged.cuh),
// captured in a CUDA graph.  FP32, complex and centered data, A = 2 or 3.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "hd_plan.h"
#include "hd_ragged.cuh"

namespace hd {

namespace {

constexpr int RT_THREADS = 256;
constexpr int kRowS2 = 4096;   // split rows of the ragged kernel: size-4096 FFTs, 16 values per thread
constexpr int kRowE = 16;
// columns per COLFWD / COLBWD tile: about 16 K elements (column x S1), so that
// the per-tile cost (queue atomic, barriers, dependency counters) is spread
// over enough independent loads per thread
__host__ __device__ constexpr int col_blk(int S1) { return S1 <= 4 ? 4096 : 16384 / S1; }

__host__ __device__ constexpr int ragged_E(int S) { return S <= 2048 ? (S < 8 ? S : 8) : 16; }

// FUSED tile: up to G = 256/T instances of one configuration.
template <int S, int KINDNB, int MULT>
__device__ __noinline__ void fused_tile(const RaggedArgs& ra, const RTile& t, unsigned char* smem) {
    using T = float2;
    constexpr int E = ragged_E(S);
    constexpr int TT = S / E;
    constexpr int KIND = KINDNB == 2 ? KIND_CENTERED : KIND_COMPLEX;
    constexpr int NB = KINDNB == 0 ? 1 : 2;
    constexpr int A = MultShape<MULT>::A;
    static_assert(MultShape<MULT>::B == 1, "single-output mults only");
    const int g = threadIdx.x / TT;
    const int tau = threadIdx.x - g * TT;
    const bool valid = g < t.count;
    const RInst& r = ra.inst[ra.order[t.first + (valid ? g : 0)]];
    ConvArgs a = conv_args_of(r);
    a.ls_pad = t.aux;
    T* st = reinterpret_cast<T*>(smem) + (size_t)g * (A * t.aux + A * FftShape<S, E>::SMEM);
    T* sm = st + A * t.aux;
    conv1d_body<float, S, E, KIND, MULT, NB, false>(a, 0, valid, tau, st, sm);
}

// columns a thread handles together in the column phases (loads in flight)
__host__ __device__ constexpr int col_u(int S1) { return S1 >= 16 ? 1 : 16 / S1 > 8 ? 8 : 16 / S1; }

template <int S1, int KIND>
__device__ __noinline__ void colfwd_tile(const RaggedArgs& ra, const RTile& t) {
    const RInst& r = ra.inst[t.first];
    const SplitArgs a = split_args_of(r);
    constexpr int CB = col_blk(S1);
    constexpr int U = col_u(S1);
    static_assert(CB % (RT_THREADS * U) == 0, "column tile");
    const int nblk = r.S2 / CB;
    const int blk = t.count % nblk;
    const int rr = (t.count / nblk) % r.n;
    const int aa = t.count / nblk / r.n;
    for (int c = (int)threadIdx.x; c < CB; c += RT_THREADS * U)
        split_colfwd_multi<float, S1, KIND, U>(a, 0, aa, rr, blk * CB + c, RT_THREADS);
}

template <int KIND, int MULT>
__device__ __noinline__ void row_tile(const RaggedArgs& ra, const RTile& t, unsigned char* smem) {
    const RInst& r = ra.inst[t.first];
    const SplitArgs a = split_args_of(r);
    split_row_body<float, kRowS2, kRowE, KIND, MULT, true>(a, t.count, true, (int)threadIdx.x,
                                                     reinterpret_cast<float2*>(smem));
}

template <int S1, int KIND>
__device__ __noinline__ void colbwd_tile(const RaggedArgs& ra, const RTile& t) {
    const RInst& r = ra.inst[t.first];
    const SplitArgs a = split_args_of(r);
    constexpr int CB = col_blk(S1);
    constexpr int U = col_u(S1) > 4 ? 4 : col_u(S1);
    static_assert(CB % (RT_THREADS * U) == 0, "column tile");
    for (int c = (int)threadIdx.x; c < CB; c += RT_THREADS * U)
        split_colbwd_multi<float, S1, KIND, false, U>(a, 0, t.count * CB + c, RT_THREADS);
    // the tile's columns of the work buffer are dead: drop them from L2
    __syncthreads();
    const float2* base = static_cast<const float2*>(a.work);
    for (int rk = 0; rk < a.n * S1; ++rk)
        l2_discard(base + (int64_t)(rk / S1) * a.S + (int64_t)(rk % S1) * a.S2 + (int64_t)t.count * CB,
                   (int64_t)CB * sizeof(float2), (int)threadIdx.x, RT_THREADS);
}

// configuration id of a FUSED tile
__host__ __device__ constexpr int fused_cfg_id(int lgS, int kindnb, int mult) { return ((lgS - 1) * 3 + kindnb) * 2 + mult; }

#define HD_FUSED_CASE(LG, KNB, ML) \
    case fused_cfg_id(LG, KNB, ML): fused_tile<(1 << LG), KNB, ML>(ra, t, smem); break;
#define HD_FUSED_LG(LG)                                                                               \
    HD_FUSED_CASE(LG, 0, 0) HD_FUSED_CASE(LG, 0, 1) HD_FUSED_CASE(LG, 1, 0) HD_FUSED_CASE(LG, 1, 1) \
    HD_FUSED_CASE(LG, 2, 0) HD_FUSED_CASE(LG, 2, 1)

__device__ void run_fused(const RaggedArgs& ra, const RTile& t, unsigned char* smem) {
    switch (t.cfg) {
        HD_FUSED_LG(3) HD_FUSED_LG(4) HD_FUSED_LG(5) HD_FUSED_LG(6) HD_FUSED_LG(7) HD_FUSED_LG(8)
        HD_FUSED_LG(9) HD_FUSED_LG(10) HD_FUSED_LG(11) HD_FUSED_LG(12)
        default: break;
    }
}

// A wait that runs out records HD_ERR_TIMEOUT and skips the tile's work, but
// the tile still signals its counter, so dependents wait at most once more.
__device__ void run_split(const RaggedArgs& ra, const RTile& t, unsigned char* smem, int* flag) {
    const RInst& r = ra.inst[t.first];
    const int kind = r.H >= 0 ? KIND_CENTERED : KIND_COMPLEX;   // H < 0 marks complex data
    if (t.type == RT_COLFWD) {
        if (r.gneed <= 0 || cta_wait(ra.gdone + r.gprev, r.gneed, ra, flag)) {
#define HD_CF(S1)                                                                          \
    case S1:                                                                               \
        if (kind == KIND_COMPLEX) colfwd_tile<S1, KIND_COMPLEX>(ra, t);                    \
        else colfwd_tile<S1, KIND_CENTERED>(ra, t);                                        \
        break;
            switch (r.S1) { HD_CF(2) HD_CF(4) HD_CF(8) HD_CF(16) default: break; }
#undef HD_CF
        }
        cta_signal(ra.cnt1 + t.first);
    } else if (t.type == RT_ROW) {
        if (cta_wait(ra.cnt1 + t.first, r.ncf + r.stall, ra, flag)) {
            if (r.A == 2) {
                if (kind == KIND_COMPLEX) row_tile<KIND_COMPLEX, MULT_PRODUCT>(ra, t, smem);
                else row_tile<KIND_CENTERED, MULT_PRODUCT>(ra, t, smem);
            } else {
                if (kind == KIND_COMPLEX) row_tile<KIND_COMPLEX, MULT_PAIRS3>(ra, t, smem);
                else row_tile<KIND_CENTERED, MULT_PAIRS3>(ra, t, smem);
            }
        }
        cta_signal(ra.cnt2 + t.first);
    } else {
        if (cta_wait(ra.cnt2 + t.first, r.nrow, ra, flag)) {
#define HD_CB(S1)                                                                          \
    case S1:                                                                               \
        if (kind == KIND_COMPLEX) colbwd_tile<S1, KIND_COMPLEX>(ra, t);                    \
        else colbwd_tile<S1, KIND_CENTERED>(ra, t);                                        \
        break;
            switch (r.S1) { HD_CB(2) HD_CB(4) HD_CB(8) HD_CB(16) default: break; }
#undef HD_CB
        }
        cta_signal(ra.gdone + r.grp);
    }
}

// Persistent loop.  Thread 0 claims the next tile while the CTA works on the
// current one, so the queue atomic is off the critical path.  A claimed tile
// only waits on earlier tiles, and the earliest unfinished tile is always
// some CTA's current tile (or the next of a CTA whose current one finished),
// so the queue always drains.
__global__ void __launch_bounds__(RT_THREADS, 1) ragged_kernel(const __grid_constant__ RaggedArgs ra) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_next, s_flag;
    if (threadIdx.x == 0) s_next = atomicAdd(ra.head, 1);
    __syncthreads();
    for (;;) {
        const int ti = s_next;
        __syncthreads();
        if (ti >= ra.ntiles) return;
        if (threadIdx.x == 0) s_next = atomicAdd(ra.head, 1);
        const RTile t = ra.tiles[ti];
        if (t.type == RT_FUSED) run_fused(ra, t, smem);
        else run_split(ra, t, smem, &s_flag);
        __syncthreads();
    }
}

int ilog2_exact(int64_t x) {
    int l = 0;
    while ((int64_t(1) << l) < x) ++l;
    return l;
}

size_t fused_group_elems(int64_t S, int A, int aux) {
    const int64_t E = ragged_E((int)S);
    (void)E;
    return (size_t)A * ((size_t)aux + (size_t)(S + (ragged_E((int)S) == 8 ? S / 8 : S / 16)));   // FftShape::SMEM
}

size_t fused_tile_smem(int64_t S, int A, int aux) {
    const int64_t T = S / ragged_E((int)S);
    const int64_t G = RT_THREADS / T;
    return (size_t)G * fused_group_elems(S, A, aux) * 8;
}

// dynamic shared memory a ragged tile may use (the kernel's own static shared
// memory and the per-block opt-in limit are checked at plan creation)
constexpr size_t kSmemMax = 226 * 1024;

// split work buffers: groups of at most kGroupBytes in a ring of kRing buffers
// (ring >= 3 keeps every wait pointing to an earlier stage of the queue)
constexpr size_t kGroupBytes = 16u << 20;
constexpr int kRing = 4;

// group size in bytes; HD_RAGGED_GROUP_MB overrides the default (tuning)
size_t group_bytes() {
    const char* e = std::getenv("HD_RAGGED_GROUP_MB");
    if (e && *e) {
        const long v = std::strtol(e, nullptr, 10);
        if (v >= 1 && v <= 4096) return (size_t)v << 20;
    }
    return kGroupBytes;
}

// ragged feasibility of a candidate for one instance
bool ragged_ok(const hd_desc* d, const hd_candidate& c) {
    const int64_t Ls = d->L[0];
    if (!single_group(d->kind, c)) return false;   // the ragged kernel runs one residue at a time
    if (c.S <= 4096) {
        if (c.S < 8 || !is_pow2(c.S)) return false;
        return fused_tile_smem(c.S, d->A, (int)staged_row(Ls)) <= kSmemMax;
    }
    return is_pow2(c.S) && c.S / kRowS2 >= 2 && c.S / kRowS2 <= 16;
}

}  // namespace

struct RaggedData {
    int64_t n = 0;
    std::vector<RInst> inst;
    std::vector<hd_candidate> cand;
    std::vector<int> kinds;            // HD_* kind of each instance
    std::vector<RTile> tiles;
    std::vector<int> order;
    RInst* d_inst = nullptr;
    RTile* d_tiles = nullptr;
    int* d_order = nullptr;
    int* d_ctr = nullptr;              // head, err, cnt1[n], cnt2[n], gdone[ngroups]
    int ngroups = 0;                   // split work-buffer groups
    void* d_work = nullptr;
    std::map<std::tuple<int64_t, int>, void*> fft_tab;
    std::map<std::tuple<int64_t, int64_t>, void*> twist_tab;
    std::map<int64_t, void*> split_tab;
    size_t smem = 0;
    int grid = 0;
    long long wait_ns = 2000000000LL;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool bound = false;
    cudaStream_t last = nullptr;
};

namespace {

void ragged_free(RaggedData* rg) {
    if (!rg) return;
    if (rg->exec) cudaGraphExecDestroy(rg->exec);
    if (rg->graph) cudaGraphDestroy(rg->graph);
    if (rg->cap) cudaStreamDestroy(rg->cap);
    for (auto& kv : rg->fft_tab) cudaFree(kv.second);
    for (auto& kv : rg->twist_tab) cudaFree(kv.second);
    for (auto& kv : rg->split_tab) cudaFree(kv.second);
    cudaFree(rg->d_inst);
    cudaFree(rg->d_tiles);
    cudaFree(rg->d_order);
    cudaFree(rg->d_ctr);
    cudaFree(rg->d_work);
    cudaGetLastError();
    delete rg;
}

hd_status choose_ragged(const hd_desc* d, hd_candidate* out) {
    std::vector<hd_candidate> cands;
    enumerate_candidates(d, &cands);
    hd_candidate tuned;
    if (cache_lookup(d, &tuned)) {
        for (auto& c : cands)
            if (c.S == tuned.S && c.n == tuned.n && ragged_ok(d, c)) {
                *out = c;
                return HD_OK;
            }
    }
    bool found = false;
    double best = 0;
    for (auto& c : cands) {
        if (!ragged_ok(d, c)) continue;
        double cost = cost_model(d->kind, d->A, d->B, c.S, c.n) * (c.S > 4096 ? 1.6 : 1.0);
        if (!found || cost < best) {
            *out = c;
            best = cost;
            found = true;
        }
    }
    return found ? HD_OK : HD_ERR_UNSUPPORTED;
}

}  // namespace

hd_status ragged_create(hd_plan** out, int64_t n, const hd_desc* descs, const hd_candidate* forced) {
    if (n <= 0 || n > (int64_t)1 << 24) return HD_ERR_INVALID;
    // the learned selector, batched over the instances it has to choose for
    std::vector<hd_candidate> sel(n);
    std::vector<char> has_sel(n, 0);
    if (!forced && selector_installed()) {
        std::vector<const hd_desc*> ds;
        std::vector<std::vector<hd_candidate>> cs;
        std::vector<int64_t> idx;
        for (int64_t i = 0; i < n; ++i) {
            const hd_desc* d = descs + i;
            hd_candidate tmp;
            if (d->m[0] != 0 || d->ndim != 1 || cache_lookup(d, &tmp)) continue;
            if (d->L[0] <= 0 || d->M[0] < hd_dealias_bound(d->kind, d->mult, d->L[0])) continue;
            std::vector<hd_candidate> all, okc;
            enumerate_candidates(d, &all);
            for (auto& c : all)
                if (ragged_ok(d, c)) okc.push_back(c);
            if (okc.empty()) continue;
            ds.push_back(d);
            cs.push_back(okc);
            idx.push_back(i);
        }
        std::vector<int> pick, conf;
        if (!ds.empty() && selector_choose_batch(ds, cs, &pick, &conf) == HD_OK) {
            const bool fb = selector_fallback() != 0;
            for (size_t k = 0; k < ds.size(); ++k) {
                hd_candidate c = cs[k][pick[k]];
                if (!conf[k] && fb) timed_choice(ds[k], ragged_ok, &c);
                sel[idx[k]] = c;
                has_sel[idx[k]] = 1;
            }
        }
    }
    RaggedData* rg = new (std::nothrow) RaggedData;
    if (!rg) return HD_ERR_NOMEM;
    rg->n = n;
    rg->inst.resize(n);
    rg->cand.resize(n);
    rg->kinds.resize(n);
    hd_status st = HD_OK;
    size_t work_total = 0;
    for (int64_t i = 0; i < n && st == HD_OK; ++i) {
        const hd_desc* d = descs + i;
        if (d->ndim != 1 || d->dtype != HD_F32 || d->B != 1 || (d->kind != HD_COMPLEX && d->kind != HD_CENTERED) ||
            !((d->mult == HD_MULT_PRODUCT && d->A == 2) || (d->mult == HD_MULT_SUM_PAIRS3 && d->A == 3)) ||
            d->L[0] <= 0 || d->M[0] <= 0 || d->flags != 0) {
            st = HD_ERR_INVALID;
            break;
        }
        if (d->M[0] < hd_dealias_bound(d->kind, d->mult, d->L[0])) {
            st = HD_ERR_ALIASED;
            break;
        }
        hd_candidate c;
        if (forced) {
            c = forced[i];
        } else if (has_sel[i]) {
            c = sel[i];
        } else if (d->m[0] > 0) {
            AxisPlan ax;
            hd_status s2 = fill_axis(d->dtype, d->kind, d->mult, d->L[0], d->M[0], d->m[0], d->p[0], d->q[0], 1, &ax);
            if (s2 != HD_OK && s2 != HD_ERR_UNSUPPORTED) {
                st = s2;
                break;
            }
            std::memset(&c, 0, sizeof(c));
            c.m = ax.m;
            c.p = ax.p;
            c.q = ax.q;
            c.S = ax.S;
            c.n = ax.n;
        } else {
            st = choose_ragged(d, &c);
            if (st != HD_OK) break;
        }
        if (!ragged_ok(d, c)) {
            st = HD_ERR_UNSUPPORTED;
            break;
        }
        c.D = 1;
        c.E = c.S <= 4096 ? ragged_E((int)c.S) : kRowE;
        c.minb = 1;
        c.comp = 0;
        rg->cand[i] = c;
        rg->kinds[i] = d->kind;
        RInst& r = rg->inst[i];
        std::memset(&r, 0, sizeof(r));
        r.L = (int)d->L[0];
        r.Ls = (int)d->L[0];
        r.H = d->kind == HD_CENTERED ? (int)(d->L[0] / 2) : -1;
        r.n = (int)c.n;
        r.N = (int)(c.n * c.S);
        r.S = (int)c.S;
        r.A = d->A;
        r.ls_pad = (int)staged_row(d->L[0]);
        r.invN = 1.0 / (double)(c.n * c.S);
        if (c.S > 4096) {
            r.S2 = kRowS2;
            r.S1 = (int)(c.S / kRowS2);
            r.ncf = d->A * r.n * (kRowS2 / col_blk(r.S1));
            r.ncb = kRowS2 / col_blk(r.S1);
            r.nrow = r.n * r.S1;
        }
    }
    if (st != HD_OK) {
        ragged_free(rg);
        return st;
    }
    // tables shared between instances
    for (int64_t i = 0; i < n && st == HD_OK; ++i) {
        RInst& r = rg->inst[i];
        const bool split = r.S > 4096;
        const int E = split ? kRowE : ragged_E(r.S);
        const int64_t Sfft = split ? kRowS2 : r.S;
        auto kf = std::make_tuple(Sfft, E);
        if (!rg->fft_tab.count(kf)) {
            void* p = nullptr;
            st = upload_fft_twiddles(Sfft, E, HD_F32, &p);
            rg->fft_tab[kf] = p;
        }
        auto kt = std::make_tuple((int64_t)r.S, (int64_t)r.n);
        if (st == HD_OK && !rg->twist_tab.count(kt)) {
            void* p = nullptr;
            st = upload_twists(r.S, r.n, HD_F32, &p);
            rg->twist_tab[kt] = p;
        }
        if (st == HD_OK && split && !rg->split_tab.count(r.S)) {
            void* p = nullptr;
            st = upload_split_twiddles(r.S1, r.S2, HD_F32, &p);
            rg->split_tab[r.S] = p;
        }
        if (st != HD_OK) break;
        r.twN = rg->twist_tab[kt];
        if (split) {
            r.twS = rg->split_tab[r.S];
            r.twS2 = rg->fft_tab[kf];
        } else {
            r.twS = rg->fft_tab[kf];
        }
    }
    // Split instances, largest work buffer first, packed into groups of at most
    // kGroupBytes; group g uses buffer g mod kRing of a ring whose total stays
    // within L2, so the work-buffer round trips between the three phases are
    // served by L2 rather than HBM.
    std::vector<int> split_ids;
    for (int64_t i = 0; i < n; ++i)
        if (rg->inst[i].S > 4096) split_ids.push_back((int)i);
    auto work_of = [&](int i) { return (size_t)rg->inst[i].A * (size_t)rg->inst[i].n * (size_t)rg->inst[i].S * 8; };
    std::stable_sort(split_ids.begin(), split_ids.end(), [&](int x, int y) { return work_of(x) > work_of(y); });
    std::vector<std::vector<int>> sgroups;
    size_t buf = 0;
    {
        const size_t gb = group_bytes();
        size_t used = 0;
        for (int i : split_ids) {
            const size_t w = work_of(i);
            if (sgroups.empty() || used + w > gb) {
                sgroups.emplace_back();
                used = 0;
            }
            sgroups.back().push_back(i);
            used += w;
            buf = std::max(buf, used);
        }
    }
    const int ng = (int)sgroups.size();
    rg->ngroups = ng;
    if (st == HD_OK && ng > 0) {
        const int ring = std::min(ng, kRing);
        work_total = buf * (size_t)ring;
        if (cudaMalloc(&rg->d_work, work_total) != cudaSuccess) {
            cudaGetLastError();
            st = HD_ERR_NOMEM;
        } else {
            for (int g = 0; g < ng; ++g) {
                size_t off = (size_t)(g % ring) * buf;
                for (int i : sgroups[g]) {
                    RInst& r = rg->inst[i];
                    r.work = static_cast<char*>(rg->d_work) + off;
                    off += work_of(i);
                    r.grp = g;
                    r.gprev = g >= ring ? g - ring : 0;
                    r.gneed = 0;
                }
            }
            // the COLFWD tiles of group g wait for all COLBWD tiles of group g - ring
            for (int g = ring; g < ng; ++g) {
                int ncb = 0;
                for (int i : sgroups[g - ring]) ncb += rg->inst[i].ncb;
                for (int i : sgroups[g]) rg->inst[i].gneed = ncb;
            }
        }
    }
    if (st != HD_OK) {
        ragged_free(rg);
        return st;
    }
    // Work queue in stages s = 0 .. ng + 1: stage s holds COLFWD of group s,
    // ROW of group s - 1 and COLBWD of group s - 2, followed by an equal share
    // of the FUSED tiles (by decreasing cost).  Every wait points to an
    // earlier stage: ROW(g) and COLBWD(g) to stage g and g + 1, COLFWD(g) to
    // COLBWD(g - ring) in stage g - ring + 2 < g for ring >= 3.
    std::vector<RTile> fused;
    size_t smem = 0;
    std::map<std::tuple<int, int>, std::vector<int>> groups;   // (cfg, n) -> instances
    for (int64_t i = 0; i < n; ++i) {
        const RInst& r = rg->inst[i];
        if (r.S > 4096) {
            smem = std::max(smem, (size_t)r.A * (kRowS2 + kRowS2 / 16) * 8);
        } else {
            const int kindnb = rg->kinds[i] == HD_CENTERED ? 2 : (r.L > r.S ? 1 : 0);
            const int cfg = fused_cfg_id(ilog2_exact(r.S), kindnb, r.A == 2 ? 0 : 1);
            groups[std::make_tuple(cfg, r.n)].push_back((int)i);
        }
    }
    std::vector<std::pair<double, RTile>> ft;
    for (auto& kv : groups) {
        auto& v = kv.second;
        std::sort(v.begin(), v.end(), [&](int x, int y) { return rg->inst[x].L > rg->inst[y].L; });
        const RInst& r0 = rg->inst[v[0]];
        const int T = r0.S / ragged_E(r0.S);
        const int G = RT_THREADS / T;
        for (size_t s = 0; s < v.size(); s += G) {
            const int cnt = (int)std::min<size_t>(G, v.size() - s);
            const int first = (int)rg->order.size();
            for (int k = 0; k < cnt; ++k) rg->order.push_back(v[s + k]);
            const int aux = rg->inst[v[s]].ls_pad;
            RTile t{RT_FUSED, std::get<0>(kv.first), first, cnt, aux, 0, 0, 0};
            smem = std::max(smem, fused_tile_smem(r0.S, r0.A, aux));
            const double cost = (double)cnt * r0.n * r0.S * std::log2((double)r0.S + 1) * (r0.A + 1);
            ft.push_back({cost, t});
        }
    }
    std::stable_sort(ft.begin(), ft.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    for (auto& x : ft) fused.push_back(x.second);
    rg->tiles.clear();
    const int nstage = ng > 0 ? ng + 2 : 0;
    size_t fpos = 0;
    for (int sg = 0; sg < nstage; ++sg) {
        if (sg < ng)
            for (int i : sgroups[sg])
                for (int c = 0; c < rg->inst[i].ncf; ++c) rg->tiles.push_back(RTile{RT_COLFWD, 0, i, c, 0, 0, 0, 0});
        if (sg >= 1 && sg - 1 < ng)
            for (int i : sgroups[sg - 1])
                for (int c = 0; c < rg->inst[i].nrow; ++c) rg->tiles.push_back(RTile{RT_ROW, 0, i, c, 0, 0, 0, 0});
        if (sg >= 2)
            for (int i : sgroups[sg - 2])
                for (int c = 0; c < rg->inst[i].ncb; ++c)
                    rg->tiles.push_back(RTile{RT_COLBWD, 0, i, c, 0, 0, 0, 0});
        const size_t upto = fused.size() * (size_t)(sg + 1) / (size_t)(nstage + 1);
        for (; fpos < upto; ++fpos) rg->tiles.push_back(fused[fpos]);
    }
    for (; fpos < fused.size(); ++fpos) rg->tiles.push_back(fused[fpos]);
    rg->smem = smem;
    if (smem > kSmemMax) {
        ragged_free(rg);
        return HD_ERR_UNSUPPORTED;
    }
    // device copies
    auto up = [&](void** dst, const void* src, size_t bytes) -> hd_status {
        if (bytes == 0) bytes = 16;
        if (cudaMalloc(dst, bytes) != cudaSuccess) {
            cudaGetLastError();
            return HD_ERR_NOMEM;
        }
        if (src && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) return HD_ERR_CUDA;
        return HD_OK;
    };
    st = up((void**)&rg->d_tiles, rg->tiles.data(), rg->tiles.size() * sizeof(RTile));
    if (st == HD_OK) st = up((void**)&rg->d_order, rg->order.data(), rg->order.size() * sizeof(int));
    if (st == HD_OK) st = up((void**)&rg->d_inst, rg->inst.data(), rg->inst.size() * sizeof(RInst));
    if (st == HD_OK) st = up((void**)&rg->d_ctr, nullptr, (size_t)(2 + 2 * n + ng) * sizeof(int));
    if (st == HD_OK) {
        // one attribute value for every ragged plan: the largest tile of any plan fits
        int dev = 0, optin = 0;
        cudaFuncAttributes fa;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (cudaFuncGetAttributes(&fa, ragged_kernel) != cudaSuccess) {
            st = HD_ERR_CUDA;
        } else {
            const size_t dynmax = (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
            if (rg->smem > dynmax) st = HD_ERR_UNSUPPORTED;
            else if (cudaFuncSetAttribute(ragged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynmax) !=
                     cudaSuccess)
                st = HD_ERR_CUDA;
        }
    }
    if (st == HD_OK) {
        int dev = 0, sms = 0, per = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, ragged_kernel, RT_THREADS, rg->smem);
        rg->grid = std::max(1, sms * std::max(1, per));
        if ((int64_t)rg->grid > (int64_t)rg->tiles.size()) rg->grid = (int)rg->tiles.size();
    }
    if (st != HD_OK) {
        cudaGetLastError();
        ragged_free(rg);
        return st;
    }
    hd_plan* pl = new (std::nothrow) hd_plan;
    if (!pl) {
        ragged_free(rg);
        return HD_ERR_NOMEM;
    }
    std::memset(pl, 0, sizeof(*pl));
    pl->ndim = 1;
    pl->dtype = HD_F32;
    pl->A = 3;
    pl->B = 1;
    pl->sticky = HD_OK;
    pl->ragged = rg;
    pl->scratch_bytes = work_total;
    cudaGetDevice(&pl->device);
    *out = pl;
    return HD_OK;
}

void ragged_destroy(hd_plan* pl) {
    ragged_free(pl->ragged);
    pl->ragged = nullptr;
}

namespace {

hd_status capture(RaggedData* rg) {
    if (rg->exec) return HD_OK;
    if (!rg->cap && cudaStreamCreateWithFlags(&rg->cap, cudaStreamNonBlocking) != cudaSuccess) return HD_ERR_CUDA;
    RaggedArgs ra;
    ra.inst = rg->d_inst;
    ra.tiles = rg->d_tiles;
    ra.order = rg->d_order;
    ra.ntiles = (int)rg->tiles.size();
    ra.head = rg->d_ctr;
    ra.err = rg->d_ctr + 1;
    ra.cnt1 = rg->d_ctr + 2;
    ra.cnt2 = rg->d_ctr + 2 + rg->n;
    ra.gdone = rg->d_ctr + 2 + 2 * rg->n;
    ra.wait_ns = rg->wait_ns;
    if (cudaStreamBeginCapture(rg->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return HD_ERR_CUDA;
    cudaMemsetAsync(rg->d_ctr, 0, (size_t)(2 + 2 * rg->n + rg->ngroups) * sizeof(int), rg->cap);
    ragged_kernel<<<rg->grid, RT_THREADS, rg->smem, rg->cap>>>(ra);
    cudaError_t e = cudaStreamEndCapture(rg->cap, &rg->graph);
    if (e != cudaSuccess) return HD_ERR_CUDA;
    if (cudaGraphInstantiate(&rg->exec, rg->graph, 0) != cudaSuccess) return HD_ERR_CUDA;
    return HD_OK;
}

}  // namespace

}  // namespace hd

using namespace hd;

extern "C" {

hd_status hd_ragged_create(hd_plan** out, int64_t n, const hd_desc* descs) {
    if (!out || !descs) return HD_ERR_INVALID;
    *out = nullptr;
    return ragged_create(out, n, descs, nullptr);
}

hd_status hd_ragged_create_candidates(hd_plan** out, int64_t n, const hd_desc* descs, const hd_candidate* c) {
    if (!out || !descs || !c) return HD_ERR_INVALID;
    *out = nullptr;
    return ragged_create(out, n, descs, c);
}

hd_status hd_ragged_bind(hd_plan* plan, const void* const* f, void* const* h) {
    if (!plan || !plan->ragged || !f || !h) return HD_ERR_INVALID;
    RaggedData* rg = plan->ragged;
    for (int64_t i = 0; i < rg->n; ++i) {
        RInst& r = rg->inst[i];
        for (int a = 0; a < 3; ++a) r.f[a] = a < r.A ? f[3 * i + a] : nullptr;
        r.h = h[i];
        for (int a = 0; a < r.A; ++a)
            if (!r.f[a]) return HD_ERR_INVALID;
        if (!r.h) return HD_ERR_INVALID;
    }
    if (cudaMemcpy(rg->d_inst, rg->inst.data(), rg->inst.size() * sizeof(RInst), cudaMemcpyHostToDevice) !=
        cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    rg->bound = true;
    return capture(rg);
}

hd_status hd_ragged_run(const hd_plan* plan, void* stream) {
    if (!plan || !plan->ragged) return HD_ERR_INVALID;
    RaggedData* rg = plan->ragged;
    if (!rg->bound || !rg->exec) return HD_ERR_INVALID;
    if (cudaGraphLaunch(rg->exec, (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    rg->last = (cudaStream_t)stream;
    return HD_OK;
}

hd_status hd_ragged_status(const hd_plan* plan) {
    if (!plan || !plan->ragged) return HD_ERR_INVALID;
    RaggedData* rg = plan->ragged;
    if (cudaStreamSynchronize(rg->last) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    int err = 0;
    if (cudaMemcpy(&err, rg->d_ctr + 1, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    return err ? HD_ERR_TIMEOUT : HD_OK;
}

hd_status hd_ragged_get_params(const hd_plan* plan, int64_t i, hd_candidate* c) {
    if (!plan || !plan->ragged || !c || i < 0 || i >= plan->ragged->n) return HD_ERR_INVALID;
    *c = plan->ragged->cand[i];
    return HD_OK;
}

hd_status hd_ragged_set_wait_limit(hd_plan* plan, int64_t ns) {
    if (!plan || !plan->ragged || ns <= 0) return HD_ERR_INVALID;
    RaggedData* rg = plan->ragged;
    rg->wait_ns = ns;
    if (rg->exec) {
        cudaGraphExecDestroy(rg->exec);
        cudaGraphDestroy(rg->graph);
        rg->exec = nullptr;
        rg->graph = nullptr;
    }
    return rg->bound ? capture(rg) : HD_OK;
}

hd_status hd_ragged_inject_stall(hd_plan* plan, int64_t i) {
    if (!plan || !plan->ragged || i < 0 || i >= plan->ragged->n) return HD_ERR_INVALID;
    RaggedData* rg = plan->ragged;
    if (rg->inst[i].S <= 4096) return HD_ERR_INVALID;
    rg->inst[i].stall = 1;
    if (cudaMemcpy(rg->d_inst + i, &rg->inst[i], sizeof(RInst), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

}  // extern "C"
