// hd_api.cu -- C ABI of libhd: plans, parameter derivation, twiddle tables,
// dispatch of the fused kernels.  Declarations and contracts: include/hd.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/hd.h"
#include "hd_dispatch.h"
#include "hd_plan.h"

using namespace hd;

// ------------------------------------------------------------------ helpers

namespace hd {

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

int64_t next_pow2_t(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

bool is_pow2(int64_t x) { return x > 0 && (x & (x - 1)) == 0; }

// zeta_N^k = exp(2 pi i k / N) in FP64.  The angle is reduced exactly to the
// first octant with integer arithmetic, so values at multiples of N/8 (and the
// symmetries between octants) are exact before rounding.
void zeta_fp64(int64_t k, int64_t N, double* c, double* s) {
    k %= N;
    if (k < 0) k += N;
    // 8k = o N + rem, o = octant
    const __int128 a = (__int128)k * 8;
    const int o = (int)(a / N);
    const int64_t rem = (int64_t)(a - (__int128)o * N);   // angle within octant: (pi/4) * rem / N
    // angle t in [0, pi/4): t = pi * rem / (4N); for odd octants use the complement
    double t;
    bool odd = (o & 1) != 0;
    if (!odd) t = M_PI * (double)rem / (4.0 * (double)N);
    else t = M_PI * (double)(N - rem) / (4.0 * (double)N);
    double ct = std::cos(t), st = std::sin(t);
    if (rem == 0) {
        ct = odd ? std::cos(M_PI / 4) : 1.0;
        st = odd ? std::sin(M_PI / 4) : 0.0;
    }
    // (x, y) of the angle o*pi/4 + t (even o) or (o+1)*pi/4 - t (odd o)
    double x, y;
    switch (o) {
        case 0: x = ct; y = st; break;             // t
        case 1: x = st; y = ct; break;             // pi/2 - t
        case 2: x = -st; y = ct; break;            // pi/2 + t
        case 3: x = -ct; y = st; break;            // pi - t
        case 4: x = -ct; y = -st; break;           // pi + t
        case 5: x = -st; y = -ct; break;           // 3pi/2 - t
        case 6: x = st; y = -ct; break;            // 3pi/2 + t
        default: x = ct; y = -st; break;           // 2pi - t
    }
    *c = x;
    *s = y;
}

// Uploads (exponent, modulus) pairs as zeta_mod^exp values, generated in FP64
// and rounded once to the plan's precision.
hd_status upload_zetas(const std::vector<std::pair<int64_t, int64_t>>& ek, int dtype, void** dev) {
    *dev = nullptr;
    const int64_t N = (int64_t)ek.size();
    if (N <= 0) return HD_ERR_INVALID;
    const size_t esz = dtype == HD_F64 ? 16 : 8;
    std::vector<unsigned char> host((size_t)N * esz);
    for (int64_t k = 0; k < N; ++k) {
        double c, s;
        zeta_fp64(ek[k].first, ek[k].second, &c, &s);
        if (dtype == HD_F64) {
            double* p = reinterpret_cast<double*>(host.data()) + 2 * k;
            p[0] = c;
            p[1] = s;
        } else {
            float* p = reinterpret_cast<float*>(host.data()) + 2 * k;
            p[0] = (float)c;
            p[1] = (float)s;
        }
    }
    void* d = nullptr;
    if (cudaMalloc(&d, host.size()) != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_NOMEM;
    }
    if (cudaMemcpy(d, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(d);
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    *dev = d;
    return HD_OK;
}

// FFT pass twiddles of a size-S FFT with E values per thread, in the layout
// of FftShape<S, E>: for each pass k with Q_k = N_k / R_k > 1, entries
// zeta_{N_k}^{c k1} at (k1 - 1) Q_k + c.
hd_status upload_fft_twiddles(int64_t S, int E, int dtype, void** dev) {
    std::vector<std::pair<int64_t, int64_t>> ek;
    int LS = 0, LE = 0;
    while ((int64_t(1) << LS) < S) ++LS;
    while ((1 << LE) < E) ++LE;
    const int KF = LE > 0 ? LS / LE : 0;
    const int K = KF + ((LE > 0 && LS % LE) ? 1 : 0);
    int64_t N = S;
    for (int k = 0; k < K; ++k) {
        const int64_t R = k < KF ? E : (int64_t(1) << (LS % LE));
        const int64_t Q = N / R;
        if (Q > 1)
            for (int64_t k1 = 1; k1 < R; ++k1)
                for (int64_t c = 0; c < Q; ++c) ek.emplace_back(c * k1, N);
        N = Q;
    }
    if (ek.empty()) ek.emplace_back(0, 1);
    return upload_zetas(ek, dtype, dev);
}

// Residue twists of an axis with n residues of size S (N = n S):
// zeta_N^{r j} at r S + j, then zeta_N^{r S} at n S + r.
hd_status upload_twists(int64_t S, int64_t n, int dtype, void** dev) {
    const int64_t N = n * S;
    std::vector<std::pair<int64_t, int64_t>> ek;
    ek.reserve((size_t)(N + n));
    for (int64_t r = 0; r < n; ++r)
        for (int64_t j = 0; j < S; ++j) ek.emplace_back(r * j, N);
    for (int64_t r = 0; r < n; ++r) ek.emplace_back(r * S, N);
    return upload_zetas(ek, dtype, dev);
}

int max_fused_S(int dtype) { return dtype == HD_F64 ? 2048 : 4096; }

int64_t split_rows(int dtype) { return max_fused_S(dtype); }

bool split_supported(int dtype, int kind, int mult, int64_t S, int nb) {
    (void)kind;
    (void)nb;
    const int64_t S2 = split_rows(dtype);
    if (!is_pow2(S) || S <= max_fused_S(dtype)) return false;
    const int64_t S1 = S / S2;
    return S1 >= 2 && S1 <= 16;
}

// zeta_S^{j2 k1} at k1 S2 + j2 (k1 < S1, j2 < S2), S = S1 S2.
hd_status upload_split_twiddles(int64_t S1, int64_t S2, int dtype, void** dev) {
    std::vector<std::pair<int64_t, int64_t>> ek;
    ek.reserve((size_t)(S1 * S2));
    for (int64_t k1 = 0; k1 < S1; ++k1)
        for (int64_t j2 = 0; j2 < S2; ++j2) ek.emplace_back(j2 * k1, S1 * S2);
    return upload_zetas(ek, dtype, dev);
}

// Transform size, residue count and folded blocks of a validated axis plan.
void axis_geometry(int kind, int64_t L, int64_t m, int64_t p, int64_t q, int64_t* S, int64_t* n, int* nb) {
    if (p == 1 && q == 1) {                    // explicit padding: one residue of size m >= M
        *S = m;
        *n = 1;
    } else if (kind == HD_COMPLEX) {
        if (p <= 2) {
            *S = m;
            *n = q;
        } else {
            *S = p * m;
            *n = q / p;
        }
    } else {
        *S = p * m / 2;
        *n = q / (p / 2);
    }
    if (kind == HD_COMPLEX) *nb = (L > *S) ? 2 : 1;
    else if (kind == HD_CENTERED) *nb = 2;
    else *nb = 1;
}

// Validates (m, p, q) of one axis; fills S, n, nb.
hd_status validate_axis(int kind, int mult, int64_t L, int64_t M, int64_t m, int64_t p, int64_t q, int64_t* S,
                        int64_t* n, int* nb) {
    if (L <= 0 || M <= 0 || m <= 0 || p <= 0 || q <= 0) return HD_ERR_INVALID;
    const int64_t bound = hd_dealias_bound(kind, mult, L);
    if (bound < 0) return HD_ERR_INVALID;
    if (M < bound) return HD_ERR_ALIASED;
    if (q * m < M) return HD_ERR_INVALID;
    if (p == 1 && q == 1) {
        if (m < M) return HD_ERR_INVALID;
    } else if (kind == HD_COMPLEX) {
        if (p * m < L) return HD_ERR_INVALID;
        if (p > 2 && q % p != 0) return HD_ERR_INVALID;
    } else {
        if (p % 2 != 0) return HD_ERR_INVALID;
        if ((p / 2) * m < (L + 1) / 2) return HD_ERR_INVALID;
        if (q % (p / 2) != 0) return HD_ERR_INVALID;
    }
    axis_geometry(kind, L, m, p, q, S, n, nb);
    if (*S * *n >= ((int64_t)1 << 31)) return HD_ERR_UNSUPPORTED;
    return HD_OK;
}

// Two CTAs per SM (128 registers) for FP32 transforms up to 2048; the
// two-output mult holds twice the residue sums and keeps 255 registers.
int default_minb(int dtype, int64_t S, int mult) {
    return (dtype == HD_F32 && S <= 2048 && mult != HD_MULT_BASDEVANT2 && mult != HD_MULT_BASDEVANT3 &&
            mult != HD_MULT_MHD3) ? 2 : 1;
}

bool fused_supported(int dtype, int kind, int mult, int64_t S, int nb, int64_t Ls, bool comp, int E, int minb) {
    if (!is_pow2(S) || S < 2 || S > max_fused_S(dtype)) return false;
    Conv1dCfg c{dtype, kind, mult, nb, (int)S, E, comp, minb};
    return conv1d_available(c, (int)staged_row(Ls));
}

bool cluster_supported(int dtype, int kind, int mult, int64_t S, int nb, int64_t Ls, int D, int E) {
    if (kind == HD_HERMITIAN || D < 2 || !is_pow2(S) || S < 2 || S > max_fused_S(dtype)) return false;
    Conv1dCfg c{dtype, kind, kernel_mult(mult), nb, (int)S, E, false, 1};
    return conv1d_cluster_available(c, (int)staged_row(Ls), D);
}

bool mult_counts_ok(int mult, int A, int B) {
    return (mult == HD_MULT_PRODUCT && A == 2 && B == 1) || (mult == HD_MULT_SUM_PAIRS3 && A == 3 && B == 1) ||
           (mult == HD_MULT_BASDEVANT2 && A == 2 && B == 2) || (mult == HD_MULT_BASDEVANT3 && A == 3 && B == 5) ||
           (mult == HD_MULT_MHD3 && A == 6 && B == 8);
}

int kernel_mult(int mult) {
    if (mult == HD_MULT_MHD3) return MULT_MHD3;
    if (mult == HD_MULT_BASDEVANT3) return MULT_BASD3;
    return mult == HD_MULT_BASDEVANT2 ? MULT_BASD2 : (mult == HD_MULT_SUM_PAIRS3 ? MULT_PAIRS3 : MULT_PRODUCT);
}

// FFT work of one convolution in units of S log2 S (model used when no
// measured timing is available): (A + B) transforms per residue, Hermitian
// residues in pairs.
double cost_model(int kind, int A, int B, int64_t S, int64_t n) {
    double lg = std::log2((double)S);
    if (lg < 1) lg = 1;
    double groups = (kind == HD_HERMITIAN) ? (double)((n + 1) / 2) : (double)n;
    return groups * (A + B) * (double)S * lg + 64.0 * groups;
}

}  // namespace hd

// ------------------------------------------------------------------ dispatch (per dtype/kind TU)

namespace hd {

#define HD_SEL(fn, c, ...)                                                                   \
    do {                                                                                     \
        if (c.mult == MULT_MHD3) {                                                           \
            if (c.dtype == HD_F32) {                                                         \
                if (c.kind == KIND_COMPLEX) return fn##_f32_complex_b8(__VA_ARGS__);         \
                if (c.kind == KIND_CENTERED) return fn##_f32_centered_b8(__VA_ARGS__);       \
                return fn##_f32_hermitian_b8(__VA_ARGS__);                                   \
            }                                                                                \
            if (c.kind == KIND_COMPLEX) return fn##_f64_complex_b8(__VA_ARGS__);             \
            if (c.kind == KIND_CENTERED) return fn##_f64_centered_b8(__VA_ARGS__);           \
            return fn##_f64_hermitian_b8(__VA_ARGS__);                                       \
        }                                                                                    \
        if (c.mult == MULT_BASD3) {                                                          \
            if (c.dtype == HD_F32) {                                                         \
                if (c.kind == KIND_COMPLEX) return fn##_f32_complex_b5(__VA_ARGS__);         \
                if (c.kind == KIND_CENTERED) return fn##_f32_centered_b5(__VA_ARGS__);       \
                return fn##_f32_hermitian_b5(__VA_ARGS__);                                   \
            }                                                                                \
            if (c.kind == KIND_COMPLEX) return fn##_f64_complex_b5(__VA_ARGS__);             \
            if (c.kind == KIND_CENTERED) return fn##_f64_centered_b5(__VA_ARGS__);           \
            return fn##_f64_hermitian_b5(__VA_ARGS__);                                       \
        }                                                                                    \
        if (c.mult == MULT_BASD2) {                                                          \
            if (c.dtype == HD_F32) {                                                         \
                if (c.kind == KIND_COMPLEX) return fn##_f32_complex_b2(__VA_ARGS__);         \
                if (c.kind == KIND_CENTERED) return fn##_f32_centered_b2(__VA_ARGS__);       \
                return fn##_f32_hermitian_b2(__VA_ARGS__);                                   \
            }                                                                                \
            if (c.kind == KIND_COMPLEX) return fn##_f64_complex_b2(__VA_ARGS__);             \
            if (c.kind == KIND_CENTERED) return fn##_f64_centered_b2(__VA_ARGS__);           \
            return fn##_f64_hermitian_b2(__VA_ARGS__);                                       \
        }                                                                                    \
        if (c.dtype == HD_F32) {                                                             \
            if (c.kind == KIND_COMPLEX) return fn##_f32_complex(__VA_ARGS__);                \
            if (c.kind == KIND_CENTERED) return fn##_f32_centered(__VA_ARGS__);              \
            return fn##_f32_hermitian(__VA_ARGS__);                                          \
        }                                                                                    \
        if (c.kind == KIND_COMPLEX) return fn##_f64_complex(__VA_ARGS__);                    \
        if (c.kind == KIND_CENTERED) return fn##_f64_centered(__VA_ARGS__);                  \
        return fn##_f64_hermitian(__VA_ARGS__);                                              \
    } while (0)

bool conv1d_available(const Conv1dCfg& c, int ls_pad) { HD_SEL(conv1d_available, c, c, ls_pad); }
int conv1d_variants(int dtype, int kind, Conv1dCfg* out, int cap) {
    Conv1dCfg c{};
    c.dtype = dtype;
    c.kind = kind;
    HD_SEL(conv1d_variants, c, out, cap);
}
cudaError_t conv1d_launch(const Conv1dCfg& c, const ConvArgs& a, cudaStream_t st) { HD_SEL(conv1d_launch, c, c, a, st); }
bool conv1d_cluster_available(const Conv1dCfg& c, int ls_pad, int D) {
    HD_SEL(conv1d_cluster_available, c, c, ls_pad, D);
}
cudaError_t conv1d_cluster_launch(const Conv1dCfg& c, const ConvArgs& a, int D, cudaStream_t st) {
    HD_SEL(conv1d_cluster_launch, c, c, a, D, st);
}
cudaError_t forward_residue_launch(const Conv1dCfg& c, const ConvArgs& a, int r, int m, void* out, cudaStream_t st) {
    HD_SEL(forward_residue_launch, c, c, a, r, m, out, st);
}

}  // namespace hd

// ------------------------------------------------------------------ C ABI

extern "C" {

hd_status hd_device_status(void) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return HD_ERR_CUDA;
    }
    const int e[24] = {conv1d_take_error_f32_complex(),     conv1d_take_error_f32_centered(),
                       conv1d_take_error_f32_hermitian(),   conv1d_take_error_f64_complex(),
                       conv1d_take_error_f64_centered(),    conv1d_take_error_f64_hermitian(),
                       conv1d_take_error_f32_complex_b2(),  conv1d_take_error_f32_centered_b2(),
                       conv1d_take_error_f32_hermitian_b2(), conv1d_take_error_f64_complex_b2(),
                       conv1d_take_error_f64_centered_b2(), conv1d_take_error_f64_hermitian_b2(),
                       conv1d_take_error_f32_complex_b5(),  conv1d_take_error_f32_centered_b5(),
                       conv1d_take_error_f32_hermitian_b5(), conv1d_take_error_f64_complex_b5(),
                       conv1d_take_error_f64_centered_b5(), conv1d_take_error_f64_hermitian_b5(),
                       conv1d_take_error_f32_complex_b8(),  conv1d_take_error_f32_centered_b8(),
                       conv1d_take_error_f32_hermitian_b8(), conv1d_take_error_f64_complex_b8(),
                       conv1d_take_error_f64_centered_b8(), conv1d_take_error_f64_hermitian_b8()};
    hd_status st = HD_OK;
    for (int v : e) {
        if (v < 0) return HD_ERR_CUDA;
        if (v > 0) st = HD_ERR_TIMEOUT;
    }
    return st;
}

const char* hd_status_string(hd_status s) {
    switch (s) {
        case HD_OK: return "HD_OK";
        case HD_ERR_INVALID: return "HD_ERR_INVALID: invalid argument";
        case HD_ERR_UNSUPPORTED: return "HD_ERR_UNSUPPORTED: shape not supported by the kernels";
        case HD_ERR_NOMEM: return "HD_ERR_NOMEM: device allocation failed";
        case HD_ERR_CUDA: return "HD_ERR_CUDA: CUDA error";
        case HD_ERR_TIMEOUT: return "HD_ERR_TIMEOUT: bounded device wait expired";
        case HD_ERR_ALIASED: return "HD_ERR_ALIASED: M is below the dealiasing bound";
        case HD_ERR_SCRATCH_LIMIT:
            return "HD_ERR_SCRATCH_LIMIT: one instance needs more work buffer than the fixed allocation-free buffer";
    }
    return "unknown hd_status";
}

hd_status hd_derive_params(int kind, int64_t L, int64_t M, int64_t m, int64_t* p, int64_t* q, int64_t* n) {
    if (L <= 0 || M <= 0 || m <= 0) return HD_ERR_INVALID;
    int64_t pp, qq, nn;
    if (kind == HD_COMPLEX) {
        pp = ceil_div(L, m);
        if (pp <= 2) {
            nn = ceil_div(M, m);
            qq = nn;
        } else {
            nn = ceil_div(M, pp * m);
            qq = nn * pp;
        }
    } else if (kind == HD_CENTERED || kind == HD_HERMITIAN) {
        pp = 2 * ceil_div(L, 2 * m);
        nn = ceil_div(2 * M, pp * m);
        qq = nn * pp / 2;
    } else {
        return HD_ERR_INVALID;
    }
    if (p) *p = pp;
    if (q) *q = qq;
    if (n) *n = nn;
    return HD_OK;
}

int64_t hd_dealias_bound(int kind, int mult, int64_t L) {
    // every output of every mult is a (signed) sum of binary products
    if (L <= 0 || (mult != HD_MULT_PRODUCT && mult != HD_MULT_SUM_PAIRS3 && mult != HD_MULT_BASDEVANT2 &&
                   mult != HD_MULT_BASDEVANT3 && mult != HD_MULT_MHD3))
        return -1;
    if (kind == HD_COMPLEX) return 2 * L - 1;
    if (kind == HD_CENTERED) return L + L / 2;
    if (kind == HD_HERMITIAN) {
        const int64_t Le = 2 * ((L + 1) / 2) - 1;
        return Le + Le / 2;
    }
    return -1;
}

hd_status hd_plan_create(hd_plan** out, int64_t L, int64_t M, int A, int B, int64_t m, int64_t p, int64_t q,
                         int D) {
    if (!out) return HD_ERR_INVALID;
    *out = nullptr;
    const int mult = B == 8 ? HD_MULT_MHD3 : (B == 5 ? HD_MULT_BASDEVANT3 : (B == 2 ? HD_MULT_BASDEVANT2 : (A == 2 ? HD_MULT_PRODUCT : HD_MULT_SUM_PAIRS3)));
    if (!hd::mult_counts_ok(mult, A, B)) return HD_ERR_INVALID;
    hd_desc d;
    std::memset(&d, 0, sizeof(d));
    d.ndim = 1;
    d.L[0] = L;
    d.M[0] = M;
    d.A = A;
    d.B = B;
    d.kind = HD_COMPLEX;
    d.dtype = HD_F32;
    d.mult = mult;
    d.m[0] = m;
    d.p[0] = p;
    d.q[0] = q;
    d.D[0] = D;
    return hd_plan_create_ex(out, &d);
}

hd_status hd_plan_create_ex(hd_plan** out, const hd_desc* d) {
    if (!out || !d) return HD_ERR_INVALID;
    *out = nullptr;
    return hd::plan_create(out, d);
}

hd_status hd_plan_get_params(const hd_plan* plan, int64_t* m, int64_t* p, int64_t* q, int* D, size_t* scratch) {
    if (!plan) return HD_ERR_INVALID;
    if (m) *m = plan->ax[0].m;
    if (p) *p = plan->ax[0].p;
    if (q) *q = plan->ax[0].q;
    if (D) *D = plan->ax[0].D;
    if (scratch) *scratch = plan->scratch_bytes;
    return HD_OK;
}

hd_status hd_convolve(const hd_plan* plan, const void* const* f, void* const* h, void* stream) {
    if (!plan) return HD_ERR_INVALID;
    return hd_convolve_batched(plan, 1, f, h, plan->instance_elems, stream);
}

hd_status hd_convolve_batched(const hd_plan* plan, int64_t count, const void* const* f, void* const* h,
                              int64_t batch_stride, void* stream) {
    if (!plan || !f || !h || count < 0) return HD_ERR_INVALID;
    if (plan->ragged) return HD_ERR_INVALID;
    if (plan->sticky != HD_OK) return plan->sticky;
    if (count == 0) return HD_OK;
    for (int a = 0; a < plan->A; ++a)
        if (!f[a]) return HD_ERR_INVALID;
    for (int b = 0; b < plan->B; ++b)
        if (!h[b]) return HD_ERR_INVALID;
    if (count > 1 && batch_stride < plan->instance_elems) return HD_ERR_INVALID;
    return hd::plan_execute(const_cast<hd_plan*>(plan), count, f, h, batch_stride, (cudaStream_t)stream);
}

hd_status hd_convolve_residues(const hd_plan* plan, int64_t r_begin, int64_t r_end, int64_t count,
                               const void* const* f, void* const* h, int64_t batch_stride, void* stream) {
    if (!plan || !f || !h || count < 0) return HD_ERR_INVALID;
    if (plan->ragged) return HD_ERR_INVALID;
    if (plan->sticky != HD_OK) return plan->sticky;
    const int64_t n = plan->ax[0].n;
    if (r_begin < 0 || r_end < r_begin || r_end > n) return HD_ERR_INVALID;
    if (count == 0) return HD_OK;
    for (int a = 0; a < plan->A; ++a)
        if (!f[a]) return HD_ERR_INVALID;
    for (int b = 0; b < plan->B; ++b)
        if (!h[b]) return HD_ERR_INVALID;
    if (count > 1 && batch_stride < plan->instance_elems) return HD_ERR_INVALID;
    const bool partial = r_begin > 0 || r_end < n;
    if (partial)
        for (int a = 0; a < plan->A; ++a)
            for (int b = 0; b < plan->B; ++b)
                if (f[a] == h[b]) return HD_ERR_INVALID;
    if (r_begin == r_end) {
        // no residue: the partial sum is zero
        hd::DeviceGuard g(plan->device);
        const size_t esz = plan->dtype == HD_F64 ? 16 : 8;
        const int64_t pitch = count > 1 ? batch_stride : plan->instance_elems;
        for (int b = 0; b < plan->B; ++b) {
            if (cudaMemset2DAsync(h[b], (size_t)pitch * esz, 0, (size_t)plan->instance_elems * esz, (size_t)count,
                                  (cudaStream_t)stream) != cudaSuccess) {
                cudaGetLastError();
                return HD_ERR_CUDA;
            }
        }
        return HD_OK;
    }
    return hd::plan_execute_range(const_cast<hd_plan*>(plan), count, f, h, batch_stride, r_begin, r_end,
                                  (cudaStream_t)stream);
}

hd_status hd_forward_residue(const hd_plan* plan, const void* f, int64_t r, void* outp, void* stream) {
    if (!plan || !f || !outp) return HD_ERR_INVALID;
    if (plan->ndim != 1 || plan->ragged) return HD_ERR_INVALID;
    if (plan->sticky != HD_OK) return plan->sticky;
    const hd::AxisPlan& ax = plan->ax[0];
    if (r < 0 || r >= ax.n) return HD_ERR_INVALID;
    if (ax.path != hd::PATH_FUSED) return HD_ERR_UNSUPPORTED;
    const void* fin[kMaxIn] = {f, f, f, f, f, f};
    ConvArgs a = hd::make_conv_args(*plan, ax, 1, fin, nullptr, 0);
    Conv1dCfg c = hd::fused_cfg(*plan, ax);
    cudaError_t e = hd::forward_residue_launch(c, a, (int)r, (int)ax.m, outp, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        const_cast<hd_plan*>(plan)->sticky = HD_ERR_CUDA;
        return HD_ERR_CUDA;
    }
    return HD_OK;
}

hd_status hd_plan_destroy(hd_plan* plan) {
    if (!plan) return HD_OK;
    hd::plan_free(plan);
    return HD_OK;
}

}  // extern "C"
