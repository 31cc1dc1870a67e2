// hd_plan.cu -- plan construction, parameter selection and execution.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "hd_plan.h"
#include "hd_split.cuh"

namespace hd {

// FP32 residue sums are compensated unless HD_COMP=0 is set in the environment.
// Compensated (TwoSum) accumulation of the residue contributions pays when
// many residues are summed: the plain FP32 sum of n terms errs by at most
// (n - 1) u relative to the sum of magnitudes, below the O(u log2 S) error of
// the FFTs themselves for n < 8.  HD_COMP=1 / HD_COMP=0 forces it on / off.
bool comp_default(int64_t n) {
    const char* e = std::getenv("HD_COMP");
    if (e && e[0] == '0') return false;
    if (e && e[0] == '1') return true;
    return n >= 8;
}

namespace {

int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// (p, q) from m for an axis when the caller leaves them at 0 (Eq. pqdef1,
// Alg. convolve / convolveX, Section 6.1-6.2); p given, q derived likewise.
void derive_pq(int kind, int64_t L, int64_t M, int64_t m, int64_t* p, int64_t* q) {
    int64_t pp = *p, qq = *q, nn;
    if (pp == 0) {
        hd_derive_params(kind, L, M, m, &pp, &qq, &nn);
        // the transform size S = p m (complex) or p m / 2 (centered, Hermitian)
        // must be a power of two: round p up (explicit padding to a longer
        // p m, which hybrid padding allows) when the paper's p gives another S
        if (kind == HD_COMPLEX && pp > 2 && !is_pow2(pp)) {
            pp = next_pow2_t(pp);
            qq = ceil_div(M, pp * m) * pp;
        } else if (kind != HD_COMPLEX && pp > 2 && !is_pow2(pp / 2)) {
            pp = 2 * next_pow2_t(pp / 2);
            qq = ceil_div(2 * M, pp * m) * (pp / 2);
        }
        if (*q != 0) qq = *q;
    } else if (qq == 0) {
        if (pp == 1 && m >= M) {
            qq = 1;
        } else if (kind == HD_COMPLEX) {
            if (pp <= 2) qq = ceil_div(M, m);
            else qq = ceil_div(M, pp * m) * pp;
        } else {
            qq = ceil_div(2 * M, pp * m) * (pp / 2);
        }
    }
    *p = pp;
    *q = qq;
}

}  // namespace

hd_status fill_axis(int dtype, int kind, int mult, int64_t L, int64_t M, int64_t m, int64_t p, int64_t q, int D,
                    AxisPlan* ax) {
    std::memset(ax, 0, sizeof(*ax));
    derive_pq(kind, L, M, m, &p, &q);
    int64_t S, n;
    int nb;
    hd_status st = validate_axis(kind, mult, L, M, m, p, q, &S, &n, &nb);
    if (st != HD_OK) return st;
    ax->kind = kind;
    ax->L = L;
    ax->M = M;
    ax->Ls = kind == HD_HERMITIAN ? (L + 1) / 2 : L;
    ax->m = m;
    ax->p = p;
    ax->q = q;
    ax->n = n;
    ax->S = S;
    ax->D = D <= 0 ? 1 : D;
    ax->nb = nb;
    ax->E = S < 8 ? (int)S : 8;
    ax->comp = dtype == HD_F32 && comp_default(n);
    ax->minb = default_minb(dtype, S, mult);
    if (fused_supported(dtype, kind, mult, S, nb, ax->Ls, ax->comp, ax->E, ax->minb)) {
        ax->path = PATH_FUSED;
        return HD_OK;
    }
    if (split_supported(dtype, kind, mult, S, nb)) {
        ax->path = PATH_SPLIT;
        ax->S2 = split_rows(dtype);
        ax->S1 = S / ax->S2;
        ax->E = 8;
        ax->minb = 1;
        return HD_OK;
    }
    return HD_ERR_UNSUPPORTED;
}


hd_status choose_axis(int dtype, int kind, int mult, int A, int B, int64_t L, int64_t M, AxisPlan* best) {
    double best_cost = 0;
    bool found = false;
    auto consider = [&](int64_t m, int64_t p, int64_t q) {
        AxisPlan ax;
        if (fill_axis(dtype, kind, mult, L, M, m, p, q, 1, &ax) != HD_OK) return;
        double c = cost_model(kind, A, B, ax.S, ax.n);
        if (ax.path == PATH_SPLIT) c *= 1.6;   // work buffer round trips through L2
        // ties (within 1%): smaller qm, then smaller m
        bool better = !found || c < best_cost * 0.99 ||
                      (c <= best_cost * 1.01 &&
                       (ax.n * ax.S < best->n * best->S || (ax.n * ax.S == best->n * best->S && ax.m < best->m)));
        if (better) {
            *best = ax;
            best_cost = c;
            found = true;
        }
    };
    for (int64_t m = 1; m <= 8192; m <<= 1) {
        consider(m, 0, 0);
        // explicit padding beyond ceil(L/m) blocks so that p m is a power of two
        int64_t p, q, n;
        hd_derive_params(kind, L, M, m, &p, &q, &n);
        if (kind == HD_COMPLEX && p > 2 && !is_pow2(p)) consider(m, next_pow2(p), 0);
        if (kind != HD_COMPLEX && p > 2 && !is_pow2(p / 2)) consider(m, 2 * next_pow2(p / 2), 0);
    }
    consider(next_pow2(M), 1, 1);   // explicit zero padding (p = q = 1)
    return found ? HD_OK : HD_ERR_UNSUPPORTED;
}

namespace {

hd_status check_desc_1d(const hd_desc* d) {
    if (d->ndim != 1) return HD_ERR_UNSUPPORTED;
    if (d->kind < HD_COMPLEX || d->kind > HD_HERMITIAN) return HD_ERR_INVALID;
    if (d->dtype != HD_F32 && d->dtype != HD_F64) return HD_ERR_INVALID;
    if (!mult_counts_ok(d->mult, d->A, d->B)) return HD_ERR_INVALID;
    if (d->L[0] <= 0 || d->M[0] <= 0 || d->m[0] < 0 || d->p[0] < 0 || d->q[0] < 0) return HD_ERR_INVALID;
    if (d->M[0] < hd_dealias_bound(d->kind, d->mult, d->L[0])) return HD_ERR_ALIASED;
    if (d->flags & ~HD_PLAN_NO_WORK_BUFFER) return HD_ERR_INVALID;
    return HD_OK;
}

// Allocates the plan for a filled axis and uploads its twiddle tables.
hd_status plan_finish(const hd_desc* d, const AxisPlan& ax, hd_plan** out) {
    hd_plan* pl = new (std::nothrow) hd_plan;
    if (!pl) return HD_ERR_NOMEM;
    std::memset(pl, 0, sizeof(*pl));
    pl->ndim = 1;
    pl->kind = d->kind;
    pl->dtype = d->dtype;
    pl->mult = d->mult;
    pl->A = d->A;
    pl->B = d->B;
    pl->sticky = HD_OK;
    pl->ax[0] = ax;
    pl->ax[0].twS = pl->ax[0].twN = nullptr;
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return HD_ERR_CUDA;
    }
    pl->instance_elems = ax.Ls;
    AxisPlan& a0 = pl->ax[0];
    a0.twS2 = nullptr;
    hd_status st;
    if (a0.path == PATH_FUSED) {
        st = upload_fft_twiddles(a0.S, a0.E, d->dtype, &a0.twS);
    } else {
        st = upload_split_twiddles(a0.S1, a0.S2, d->dtype, &a0.twS);
        if (st == HD_OK) st = upload_fft_twiddles(a0.S2, a0.E, d->dtype, &a0.twS2);
        if (st == HD_OK) {
            // work buffer of Section 5: max(A, B) n S values per instance (the
            // rows write output b over part b), a chunk of instances at a time,
            // at most 64 MiB so that the round trips between the three phases
            // stay in L2
            const size_t esz = d->dtype == HD_F64 ? 16 : 8;
            const size_t per = (size_t)(d->A > d->B ? d->A : d->B) * (size_t)split_block(a0) * (size_t)a0.S * esz;
            int64_t ch = (int64_t)((64u << 20) / per);
            if (ch > 2048) ch = 2048;
            if (ch < 1) ch = 1;
            a0.chunk = ch;
            pl->scratch_bytes = (d->flags & HD_PLAN_NO_WORK_BUFFER) ? 0 : per * (size_t)ch;
            if (pl->scratch_bytes && cudaMalloc(&pl->scratch, pl->scratch_bytes) != cudaSuccess) {
                cudaGetLastError();
                pl->scratch = nullptr;
                st = HD_ERR_NOMEM;
            }
        }
    }
    if (st == HD_OK) st = upload_twists(a0.S, a0.n, d->dtype, &a0.twN);
    if (st != HD_OK) {
        plan_free(pl);
        return st;
    }
    *out = pl;
    return HD_OK;
}

}  // namespace

// Axis parameters of a 1D description from a candidate (m, p, q, D, variant).
hd_status axis_from_candidate(const hd_desc* d, const hd_candidate* c, AxisPlan* ax) {
    hd_status st = fill_axis(d->dtype, d->kind, d->mult, d->L[0], d->M[0], c->m, c->p, c->q, c->D, ax);
    if (st != HD_OK && st != HD_ERR_UNSUPPORTED) return st;
    if (ax->S != c->S || ax->n != c->n) return HD_ERR_INVALID;
    ax->comp = c->comp != 0 && d->dtype == HD_F32;
    if (ax->path == PATH_FUSED && c->D > 1 && d->kind != HD_HERMITIAN) {   // residue groups on a cluster
        if (!cluster_supported(d->dtype, d->kind, d->mult, ax->S, ax->nb, ax->Ls, c->D, c->E) || c->D > ax->n)
            return HD_ERR_UNSUPPORTED;
        ax->E = c->E;
        ax->minb = 1;
        ax->comp = false;
        return HD_OK;
    }
    if (ax->path == PATH_FUSED) {
        ax->E = c->E;
        ax->minb = c->minb;
        if (!fused_supported(d->dtype, d->kind, d->mult, ax->S, ax->nb, ax->Ls, ax->comp, ax->E, ax->minb))
            return HD_ERR_UNSUPPORTED;
    }
    return HD_OK;
}

// Parameters of a 1D axis given with m = 0: the tuning cache, else the learned
// selector (the timed search instead when it is unsure and its fallback is on),
// else the cost model.  Also used for the innermost axis of N-D plans.
hd_status auto_axis(const hd_desc* d, AxisPlan* ax) {
    hd_candidate c;
    if (cache_lookup(d, &c) && axis_from_candidate(d, &c, ax) == HD_OK) return HD_OK;
    if (selector_installed() && d->B == 1) {   // trained on single-output mults
        std::vector<hd_candidate> all, cands;
        enumerate_candidates(d, &all);
        for (auto& x : all)
            if (single_group(d->kind, x)) cands.push_back(x);
        std::vector<int> pick, conf;
        if (!cands.empty() && selector_choose_batch({d}, {cands}, &pick, &conf) == HD_OK) {
            c = cands[pick[0]];
            if (!conf[0] && selector_fallback()) timed_choice(d, nullptr, &c);
            if (axis_from_candidate(d, &c, ax) == HD_OK) return HD_OK;
        }
    }
    return choose_axis(d->dtype, d->kind, d->mult, d->A, d->B, d->L[0], d->M[0], ax);
}

hd_status plan_create_from(hd_plan** out, const hd_desc* d, const hd_candidate* c) {
    hd_status st = check_desc_1d(d);
    if (st != HD_OK) return st;
    AxisPlan ax;
    st = axis_from_candidate(d, c, &ax);
    if (st != HD_OK) return st;
    return plan_finish(d, ax, out);
}

hd_status plan_create(hd_plan** out, const hd_desc* d) {
    if (d->ndim == 2 || d->ndim == 3) return plan_create_nd(out, d);
    hd_status st = check_desc_1d(d);
    if (st != HD_OK) return st;
    AxisPlan ax;
    if (d->m[0] == 0) st = auto_axis(d, &ax);
    else st = fill_axis(d->dtype, d->kind, d->mult, d->L[0], d->M[0], d->m[0], d->p[0], d->q[0], d->D[0], &ax);
    if (st != HD_OK) return st;
    if (d->D[0] > 0) ax.D = d->D[0];
    if (ax.D > 1 && d->kind != HD_HERMITIAN && ax.path == PATH_FUSED) {   // D residue groups at once: the cluster variant
        const int ce = cluster_default_E(d->dtype, ax.S);
        if (ax.D > ax.n || !cluster_supported(d->dtype, d->kind, d->mult, ax.S, ax.nb, ax.Ls, ax.D, ce))
            return HD_ERR_UNSUPPORTED;
        ax.E = ce;
        ax.minb = 1;
        ax.comp = false;
    }
    return plan_finish(d, ax, out);
}

ConvArgs make_conv_args(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f, void* const* h,
                        int64_t stride) {
    ConvArgs a;
    std::memset(&a, 0, sizeof(a));
    for (int i = 0; i < pl.A && i < kMaxIn; ++i) a.f[i] = f[i];
    for (int b = 0; b < pl.B && b < kMaxOut; ++b) a.h[b] = h ? h[b] : nullptr;
    a.stride = stride;
    a.count = count;
    a.L = (int)ax.L;
    a.Ls = (int)ax.Ls;
    a.H = (int)(ax.L / 2);
    a.n = (int)ax.n;
    a.N = (int)(ax.n * ax.S);
    a.ls_pad = (int)staged_row(ax.Ls);
    a.twS = ax.twS;
    a.twN = ax.twN;
    a.invN = 1.0 / (double)(ax.n * ax.S);
    a.r_begin = 0;
    a.r_end = (int)ax.n;
    return a;
}

Conv1dCfg fused_cfg(const hd_plan& pl, const AxisPlan& ax) {
    Conv1dCfg c;
    c.dtype = pl.dtype;
    c.kind = ax.kind;
    c.mult = kernel_mult(pl.mult);
    c.nb = ax.nb;
    c.S = (int)ax.S;
    c.E = ax.E;
    c.comp = ax.comp;
    c.minb = ax.minb;
    return c;
}

SplitArgs make_split_args(const hd_plan& pl, const AxisPlan& ax, int64_t first, int64_t count, const void* const* f,
                          void* const* h, int64_t stride, void* work) {
    SplitArgs a;
    std::memset(&a, 0, sizeof(a));
    const size_t esz = pl.dtype == HD_F64 ? 16 : 8;
    for (int i = 0; i < pl.A && i < kMaxIn; ++i) a.f[i] = static_cast<const char*>(f[i]) + first * stride * esz;
    for (int b = 0; b < pl.B && b < kMaxOut; ++b) a.h[b] = static_cast<char*>(h[b]) + first * stride * esz;
    a.stride = stride;
    a.count = count;
    a.L = (int)ax.L;
    a.Ls = (int)ax.Ls;
    a.H = (int)(ax.L / 2);
    a.n = (int)ax.n;
    a.S = (int)ax.S;
    a.S1 = (int)ax.S1;
    a.S2 = (int)ax.S2;
    a.A = pl.A;
    a.B = pl.B;
    a.P = pl.A > pl.B ? pl.A : pl.B;
    a.twS = ax.twS;
    a.twR = ax.twN;
    a.twS2 = ax.twS2;
    a.work = work;
    a.invN = 1.0 / (double)(ax.n * ax.S);
    a.r0 = 0;
    a.nr = (int)ax.n;
    a.accumulate = 0;
    return a;
}

hd_status split_execute(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f, void* const* h,
                        int64_t stride, void* work, int64_t chunk, cudaStream_t st) {
    return split_execute_range(pl, ax, count, f, h, stride, work, chunk, 0, ax.n, st);
}

hd_status split_execute_range(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f,
                              void* const* h, int64_t stride, void* work, int64_t chunk, int64_t r_begin,
                              int64_t r_end, cudaStream_t st) {
    const int mult = kernel_mult(pl.mult);
    const int64_t blk = split_block(ax);
    // residue blocks re-read the inputs after the first block has written the
    // output, so blocked plans cannot write over their inputs
    if (r_begin + blk < r_end)
        for (int a = 0; a < pl.A; ++a)
            for (int b = 0; b < pl.B; ++b)
                if (f[a] == h[b]) return HD_ERR_INVALID;
    for (int64_t first = 0; first < count; first += chunk) {
        const int64_t cnt = count - first < chunk ? count - first : chunk;
        SplitArgs a = make_split_args(pl, ax, first, cnt, f, h, stride, work);
        for (int64_t r0 = r_begin; r0 < r_end; r0 += blk) {
            a.r0 = (int)r0;
            a.nr = (int)(r_end - r0 < blk ? r_end - r0 : blk);
            a.accumulate = r0 > r_begin;
            cudaError_t e = pl.dtype == HD_F64 ? split_launch_f64(a, ax.kind, mult, ax.comp, st)
                                               : split_launch_f32(a, ax.kind, mult, ax.comp, st);
            if (e != cudaSuccess) return HD_ERR_CUDA;
        }
    }
    return HD_OK;
}

hd_status rows_execute(const hd_plan& pl, const AxisPlan& ax, int64_t count, const void* const* f,
                       void* const* h, int64_t stride, void* scratch, cudaStream_t st) {
    if (ax.path == PATH_SPLIT) return split_execute(pl, ax, count, f, h, stride, scratch, ax.chunk, st);
    ConvArgs a = make_conv_args(pl, ax, count, f, h, stride);
    return conv1d_launch(fused_cfg(pl, ax), a, st) == cudaSuccess ? HD_OK : HD_ERR_CUDA;
}

hd_status plan_execute(hd_plan* pl, int64_t count, const void* const* f, void* const* h, int64_t stride,
                       cudaStream_t st) {
    return plan_execute_range(pl, count, f, h, stride, 0, pl->ax[0].n, st);
}

hd_status plan_execute_range(hd_plan* pl, int64_t count, const void* const* f, void* const* h, int64_t stride,
                             int64_t r_begin, int64_t r_end, cudaStream_t st) {
    DeviceGuard g(pl->device);
    if (pl->ndim > 1) {
        hd_status s2 = plan_execute_nd(pl, count, f, h, stride, r_begin, r_end, st);
        if (s2 != HD_OK) pl->sticky = s2;
        return s2;
    }
    const AxisPlan& ax = pl->ax[0];
    if (ax.path == PATH_SPLIT) {
        if (!pl->scratch) return HD_ERR_UNSUPPORTED;   // created without a work buffer
        hd_status s2 = split_execute_range(*pl, ax, count, f, h, stride, pl->scratch, ax.chunk, r_begin, r_end, st);
        if (s2 == HD_ERR_CUDA) pl->sticky = s2;
        return s2;
    }
    ConvArgs a = make_conv_args(*pl, ax, count, f, h, stride);
    a.r_begin = (int)r_begin;
    a.r_end = (int)r_end;
    const bool cluster = ax.D > 1 && ax.kind != HD_HERMITIAN;
    cudaError_t e = cluster ? conv1d_cluster_launch(fused_cfg(*pl, ax), a, ax.D, st)
                            : conv1d_launch(fused_cfg(*pl, ax), a, st);
    if (e != cudaSuccess) {
        pl->sticky = HD_ERR_CUDA;
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

void plan_free(hd_plan* pl) {
    if (!pl) return;
    DeviceGuard g(pl->device);
    cudaDeviceSynchronize();
    if (pl->ragged) ragged_destroy(pl);
    for (int i = 0; i < 3; ++i) {
        if (pl->ax[i].twS) cudaFree(pl->ax[i].twS);
        if (pl->ax[i].twN) cudaFree(pl->ax[i].twN);
        if (pl->ax[i].twS2) cudaFree(pl->ax[i].twS2);
    }
    for (int i = 0; i < 2; ++i)
        if (pl->work[i]) cudaFree(pl->work[i]);
    if (pl->scratch) cudaFree(pl->scratch);
    cudaGetLastError();
    delete pl;
}

}  // namespace hd
