// hd_nd.cu -- multidimensional convolutions by the paper's decomposition
// (Section 5): residue transforms along the outer axis, lower-dimensional
// sub-convolutions of the transformed slices, and inverse transforms along the
// outer axis, recursively; the innermost axis is a batch of 1D convolutions.
// Hermitian data (Section 5, last paragraphs): outer axes centered, innermost
// axis Hermitian, only its non-negative half stored and transformed.
#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <new>

#include "hd_cols.cuh"
#include "hd_plan.h"

namespace hd {

namespace {

int col_E_of(int dtype, int64_t S) { return dtype == HD_F64 ? col_E_of_f64((int)S) : col_E_of_f32((int)S); }

// Work buffer of an inner outer level (the middle axis of a 3D plan): no
// limit by default (all of the level's instances in one pass).  HD_ND_CHUNK_MB
// limits it to that many MiB, in chunks of the level's instances: the chunk's
// round trips then stay in L2 and the plan needs less memory, but the smaller
// launches were measured slower on the 256^3 Hermitian plan (1,143 conv/s at
// 24 MiB, 1,300 at 64 MiB, against 1,440 without a limit).
size_t level_chunk_bytes() {
    const char* e = std::getenv("HD_ND_CHUNK_MB");
    if (e && *e) {
        const long v = std::strtol(e, nullptr, 10);
        if (v >= 1 && v <= 4096) return (size_t)v << 20;
    }
    return (size_t)1 << 62;
}

bool col_supported(int dtype, int64_t S) { return is_pow2(S) && S >= 2 && S <= max_fused_S(dtype); }

// Outer-axis parameters: the cost-model choice among legal m with a supported
// column transform, or the caller's (m, p, q).
hd_status outer_axis(int dtype, int kind, int mult, int A, int B, int64_t L, int64_t M, int64_t m, int64_t p, int64_t q,
                     AxisPlan* ax) {
    if (m > 0) {
        hd_status st = fill_axis(dtype, kind, mult, L, M, m, p, q, 1, ax);
        if (st != HD_OK && st != HD_ERR_UNSUPPORTED) return st;
        if (!col_supported(dtype, ax->S)) return HD_ERR_UNSUPPORTED;
        return HD_OK;
    }
    bool found = false;
    double best = 0;
    auto consider = [&](int64_t mm, int64_t pp, int64_t qq) {
        AxisPlan cand;
        const hd_status s2 = fill_axis(dtype, kind, mult, L, M, mm, pp, qq, 1, &cand);
        if (s2 != HD_OK && s2 != HD_ERR_UNSUPPORTED) return;
        if (!col_supported(dtype, cand.S)) return;
        const double c = cost_model(kind, A, B, cand.S, cand.n);
        if (!found || c < best * 0.99 || (c <= best * 1.01 && cand.n * cand.S < ax->n * ax->S)) {
            *ax = cand;
            best = c;
            found = true;
        }
    };
    auto np2 = [](int64_t x) {
        int64_t t = 1;
        while (t < x) t <<= 1;
        return t;
    };
    for (int64_t mm = 1; mm <= 8192; mm <<= 1) {
        int64_t pp, qq, nn;
        if (hd_derive_params(kind, L, M, mm, &pp, &qq, &nn) != HD_OK) continue;
        consider(mm, 0, 0);
        if (kind == HD_COMPLEX && pp > 2 && !is_pow2(pp)) consider(mm, np2(pp), 0);
        if (kind != HD_COMPLEX && pp > 2 && !is_pow2(pp / 2)) consider(mm, 2 * np2(pp / 2), 0);
    }
    consider(np2(M), 1, 1);
    return found ? HD_OK : HD_ERR_UNSUPPORTED;
}

ColArgs make_col_args(const hd_plan& pl, const AxisPlan& ax, int level, int64_t cnt, int64_t inst_stride,
                      int64_t ncols, int r0, int nr) {
    ColArgs a;
    std::memset(&a, 0, sizeof(a));
    a.inst_stride = inst_stride;
    a.count = cnt;
    a.pitch = ncols;
    a.ncols = ncols;
    a.L = (int)ax.L;
    a.H = (int)(ax.L / 2);
    a.n = (int)ax.n;
    a.S = (int)ax.S;
    a.A = pl.A;
    a.B = pl.B;
    a.r0 = r0;
    a.nr = nr;
    a.twS = ax.twS;
    a.twN = ax.twN;
    a.invN = 1.0 / (double)(ax.n * ax.S);
    a.work = pl.work[level];
    return a;
}

int64_t ncols_of(const hd_plan& pl, int level) {
    int64_t c = 1;
    for (int i = level + 1; i < pl.ndim; ++i) c *= pl.ax[i].Ls;
    return c;
}

hd_status exec_level(const hd_plan& pl, int level, int64_t cnt, const void* const* f, int64_t inst_stride,
                     void* const* h, int64_t r_begin, int64_t r_end, cudaStream_t st);

// One pass of outer level `level` over `cnt` instances (at most the level's
// chunk): residue transforms along the axis, the sub-convolutions of the
// transformed slices, inverse transforms.  Residues r_begin <= r < r_end of
// the axis only (the partial sums of a residue-sharded convolution, on the
// outermost axis; every residue on the inner ones).
hd_status exec_level_pass(const hd_plan& pl, int level, int64_t cnt, const void* const* f, int64_t inst_stride,
                          void* const* h, int64_t r_begin, int64_t r_end, cudaStream_t st) {
    const AxisPlan& ax = pl.ax[level];
    const int64_t ncols = ncols_of(pl, level);
    const size_t esz = pl.dtype == HD_F64 ? 16 : 8;
    const int nr = ax.D > 0 && ax.D < ax.n ? ax.D : (int)ax.n;
    const int outer_kind = ax.kind == HD_COMPLEX ? KIND_COMPLEX : KIND_CENTERED;
    for (int r0 = (int)r_begin; r0 < r_end; r0 += nr) {
        const int nrb = (int)(r_end - r0 < nr ? r_end - r0 : nr);
        ColArgs a = make_col_args(pl, ax, level, cnt, inst_stride, ncols, r0, nrb);
        for (int i = 0; i < pl.A; ++i) a.f[i] = f[i];
        cudaError_t e = pl.dtype == HD_F64 ? col_launch_f64(a, outer_kind, false, true, st)
                                           : col_launch_f32(a, outer_kind, false, true, st);
        if (e != cudaSuccess) return HD_ERR_CUDA;
        // the transformed slices: A batches of cnt * nrb * S sub-arrays of ncols
        // values; the sub-convolutions write output b over part b
        const int64_t sub = cnt * nrb * ax.S;
        const void* g[kMaxIn];
        void* gh[kMaxOut];
        for (int i = 0; i < pl.A; ++i) g[i] = static_cast<const char*>(pl.work[level]) + (size_t)i * sub * ncols * esz;
        for (int b = 0; b < pl.B; ++b) gh[b] = static_cast<char*>(pl.work[level]) + (size_t)b * sub * ncols * esz;
        hd_status s2 = exec_level(pl, level + 1, sub, g, ncols, gh, 0, pl.ax[level + 1].n, st);
        if (s2 != HD_OK) return s2;
        for (int b = 0; b < pl.B; ++b) a.h[b] = h[b];
        a.accumulate = r0 > r_begin;
        e = pl.dtype == HD_F64 ? col_launch_f64(a, outer_kind, false, false, st)
                               : col_launch_f32(a, outer_kind, false, false, st);
        if (e != cudaSuccess) return HD_ERR_CUDA;
    }
    return HD_OK;
}

// Convolves `cnt` instances of the sub-array of axes level..ndim-1: A inputs
// f, B outputs h.  The instances of an outer level are independent, so a level
// whose work buffer for all of them would not stay in L2 runs them in chunks
// (the level's chunk), each chunk's forward transforms, sub-convolutions and
// inverse transforms while its work buffer is L2-resident.
hd_status exec_level(const hd_plan& pl, int level, int64_t cnt, const void* const* f, int64_t inst_stride,
                     void* const* h, int64_t r_begin, int64_t r_end, cudaStream_t st) {
    const AxisPlan& ax = pl.ax[level];
    if (level == pl.ndim - 1) return rows_execute(pl, ax, cnt, f, h, inst_stride, pl.scratch, st);
    const size_t esz = pl.dtype == HD_F64 ? 16 : 8;
    const int64_t ch = pl.level_chunk[level] > 0 ? pl.level_chunk[level] : cnt;
    for (int64_t c0 = 0; c0 < cnt; c0 += ch) {
        const int64_t cc = cnt - c0 < ch ? cnt - c0 : ch;
        const void* fc[kMaxIn];
        void* hc[kMaxOut];
        for (int a = 0; a < pl.A; ++a) fc[a] = static_cast<const char*>(f[a]) + (size_t)(c0 * inst_stride) * esz;
        for (int b = 0; b < pl.B; ++b) hc[b] = static_cast<char*>(h[b]) + (size_t)(c0 * inst_stride) * esz;
        hd_status s2 = exec_level_pass(pl, level, cc, fc, inst_stride, hc, r_begin, r_end, st);
        if (s2 != HD_OK) return s2;
    }
    return HD_OK;
}

}  // namespace

hd_status plan_create_nd(hd_plan** out, const hd_desc* d) {
    const int nd = d->ndim;
    if (d->kind < HD_COMPLEX || d->kind > HD_HERMITIAN) return HD_ERR_INVALID;
    if (d->dtype != HD_F32 && d->dtype != HD_F64) return HD_ERR_INVALID;
    if (!mult_counts_ok(d->mult, d->A, d->B)) return HD_ERR_INVALID;
    if (d->flags & ~HD_PLAN_NO_WORK_BUFFER) return HD_ERR_INVALID;
    if (d->flags) return HD_ERR_UNSUPPORTED;
    for (int i = 0; i < nd; ++i) {
        if (d->L[i] <= 0 || d->M[i] <= 0 || d->m[i] < 0 || d->p[i] < 0 || d->q[i] < 0 || d->D[i] < 0)
            return HD_ERR_INVALID;
        if (d->row_pitch[i] != 0) return HD_ERR_UNSUPPORTED;   // packed layouts only
        const int k = i < nd - 1 ? (d->kind == HD_COMPLEX ? HD_COMPLEX : HD_CENTERED) : d->kind;
        if (d->M[i] < hd_dealias_bound(k, d->mult, d->L[i])) return HD_ERR_ALIASED;
    }
    hd_plan* pl = new (std::nothrow) hd_plan;
    if (!pl) return HD_ERR_NOMEM;
    std::memset(pl, 0, sizeof(*pl));
    pl->ndim = nd;
    pl->kind = d->kind;
    pl->dtype = d->dtype;
    pl->mult = d->mult;
    pl->A = d->A;
    pl->B = d->B;
    pl->sticky = HD_OK;
    if (cudaGetDevice(&pl->device) != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return HD_ERR_CUDA;
    }
    hd_status st = HD_OK;
    for (int i = 0; i < nd && st == HD_OK; ++i) {
        AxisPlan& ax = pl->ax[i];
        if (i < nd - 1) {
            const int k = d->kind == HD_COMPLEX ? HD_COMPLEX : HD_CENTERED;
            st = outer_axis(d->dtype, k, d->mult, d->A, d->B, d->L[i], d->M[i], d->m[i], d->p[i], d->q[i], &ax);
            if (st == HD_OK) {
                ax.path = PATH_COLUMN;
                ax.E = col_E_of(d->dtype, ax.S);
                ax.comp = false;
                ax.D = d->D[i] > 0 ? d->D[i] : (int)ax.n;
                // a middle axis writes its outputs over its inputs in the parent's work
                // buffer, so all of its residues must be read before the first is written
                if (i > 0 && ax.D < ax.n) st = HD_ERR_UNSUPPORTED;
            }
        } else if (d->m[i] == 0) {
            // the innermost axis is a batch of 1D convolutions: tuning cache, selector, cost model
            hd_desc d1;
            std::memset(&d1, 0, sizeof(d1));
            d1.ndim = 1;
            d1.L[0] = d->L[i];
            d1.M[0] = d->M[i];
            d1.A = d->A;
            d1.B = d->B;
            d1.kind = d->kind;
            d1.dtype = d->dtype;
            d1.mult = d->mult;
            st = auto_axis(&d1, &ax);
        } else {
            st = fill_axis(d->dtype, d->kind, d->mult, d->L[i], d->M[i], d->m[i], d->p[i], d->q[i], d->D[i], &ax);
        }
    }
    if (st != HD_OK) {
        delete pl;
        return st;
    }
    for (int i = 0; i < nd; ++i) {
        AxisPlan& ax = pl->ax[i];
        ax.twS = ax.twN = ax.twS2 = nullptr;
    }
    // tables
    for (int i = 0; i < nd && st == HD_OK; ++i) {
        AxisPlan& ax = pl->ax[i];
        if (ax.path == PATH_SPLIT) {
            st = upload_split_twiddles(ax.S1, ax.S2, d->dtype, &ax.twS);
            if (st == HD_OK) st = upload_fft_twiddles(ax.S2, ax.E, d->dtype, &ax.twS2);
        } else {
            st = upload_fft_twiddles(ax.S, ax.E, d->dtype, &ax.twS);
        }
        if (st == HD_OK) st = upload_twists(ax.S, ax.n, d->dtype, &ax.twN);
    }
    // work buffers: level k holds max(A, B) * chunk_k * D_k * S_k * ncols_k values, where
    // chunk_k <= count_k (count_0 = 1) keeps the buffer of an inner outer level within
    // level_chunk_bytes(), so that its round trips between the kernels stay in L2
    int64_t inst = 1;
    pl->instance_elems = 1;
    for (int i = 0; i < nd; ++i) pl->instance_elems *= pl->ax[i].Ls;
    const size_t esz = d->dtype == HD_F64 ? 16 : 8;
    for (int k = 0; k < nd - 1 && st == HD_OK; ++k) {
        const AxisPlan& ax = pl->ax[k];
        const int64_t nr = ax.D;
        const int64_t per = (int64_t)(d->A > d->B ? d->A : d->B) * nr * ax.S * ncols_of(*pl, k);   // per instance
        int64_t chunk = inst;
        if (k > 0) {
            const int64_t cap = (int64_t)(level_chunk_bytes() / ((size_t)per * esz));
            chunk = cap < 1 ? 1 : (cap < inst ? cap : inst);
        }
        pl->level_chunk[k] = chunk;
        const int64_t elems = per * chunk;
        if (inst * nr * ax.S > 65535 * 64) {
            st = HD_ERR_UNSUPPORTED;
            break;
        }
        if (cudaMalloc(&pl->work[k], (size_t)elems * esz) != cudaSuccess) {
            cudaGetLastError();
            pl->work[k] = nullptr;
            st = HD_ERR_NOMEM;
            break;
        }
        pl->scratch_bytes += (size_t)elems * esz;
        inst *= nr * ax.S;
    }
    // the sub-convolutions write their outputs over their inputs, which residue
    // blocks of the split path would read again after the first block
    if (st == HD_OK && pl->ax[nd - 1].path == PATH_SPLIT && split_block(pl->ax[nd - 1]) < pl->ax[nd - 1].n)
        st = HD_ERR_UNSUPPORTED;
    // the innermost rows of the split path use the plan's chunked work buffer
    if (st == HD_OK && pl->ax[nd - 1].path == PATH_SPLIT) {
        AxisPlan& ax = pl->ax[nd - 1];
        const size_t per = (size_t)(d->A > d->B ? d->A : d->B) * (size_t)split_block(ax) * (size_t)ax.S * esz;
        int64_t ch = (int64_t)((64u << 20) / per);   // as 1D plans: at most 64 MiB, L2-resident
        ax.chunk = ch < 1 ? 1 : (ch > 2048 ? 2048 : ch);
        if (cudaMalloc(&pl->scratch, per * (size_t)ax.chunk) != cudaSuccess) {
            cudaGetLastError();
            pl->scratch = nullptr;
            st = HD_ERR_NOMEM;
        } else {
            pl->scratch_bytes += per * (size_t)ax.chunk;
        }
    }
    if (st != HD_OK) {
        plan_free(pl);
        return st;
    }
    *out = pl;
    return HD_OK;
}

hd_status plan_execute_nd(hd_plan* pl, int64_t count, const void* const* f, void* const* h, int64_t stride,
                          int64_t r_begin, int64_t r_end, cudaStream_t st) {
    const size_t esz = pl->dtype == HD_F64 ? 16 : 8;
    for (int64_t i = 0; i < count; ++i) {
        const void* fi[kMaxIn];
        void* hi[kMaxOut];
        for (int a = 0; a < pl->A; ++a) fi[a] = static_cast<const char*>(f[a]) + (size_t)(i * stride) * esz;
        for (int b = 0; b < pl->B; ++b) hi[b] = static_cast<char*>(h[b]) + (size_t)(i * stride) * esz;
        hd_status s2 = exec_level(*pl, 0, 1, fi, pl->instance_elems, hi, r_begin, r_end, st);
        if (s2 != HD_OK) return s2;
    }
    return HD_OK;
}

}  // namespace hd

extern "C" hd_status hd_plan_get_axis_params(const hd_plan* plan, int axis, int64_t* m, int64_t* p, int64_t* q,
                                             int* D, int64_t* S, int64_t* n) {
    if (!plan || axis < 0 || axis >= plan->ndim) return HD_ERR_INVALID;
    const hd::AxisPlan& ax = plan->ax[axis];
    if (m) *m = ax.m;
    if (p) *p = ax.p;
    if (q) *q = ax.q;
    if (D) *D = ax.D;
    if (S) *S = ax.S;
    if (n) *n = ax.n;
    return HD_OK;
}
