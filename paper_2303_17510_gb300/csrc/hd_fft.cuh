// hd_fft.cuh -- block-level radix-E FFT engine for sm_103a.
//
// One thread group of T = S/E threads computes one size-S FFT (S a power of
// two).  Each thread keeps E values in registers; passes are radix-E
// butterflies in registers (a final smaller radix when log2 S is not a
// multiple of log2 E), and between passes the group exchanges values through
// shared memory.  This is the size-m FFT of the method (Section 2: the
// unpadded FFTs the residue transforms call; Section 6.1: for p > 2 the
// size-p DFTs along t and the size-m FFTs along s form one size-pm FFT).
//
// Sign convention (Section 2): the forward transform is
//     X_k = sum_j zeta_S^{k j} x_j,   zeta_S = exp(+2 pi i / S),
// the inverse is the unnormalized sum with zeta^{-}.
//
// Data layouts
//   natural   thread tau holds x[tau + T e] in register e  (forward input,
//             inverse output)
//   spectral  thread tau holds X[tau + T beta + (S/R_last) k1] in register
//             beta*R_last + k1, where R_last is the radix of the last pass
//             (forward output, inverse input).  Pointwise `mult` works in this
//             layout directly: every spectrum of one size has the same map.
//
// Pass k (sub-transform size N_k = S / prod_{i<k} R_i, Q_k = N_k / R_k)
// acts on virtual threads nu = tau + T beta (beta < E/R_k), nu = b Q_k + c:
// an R_k-point DFT over the R_k values of sub-problem b at c + i Q_k, then
// the twiddle zeta_{N_k}^{c k1}.  Result k1 of nu goes to shared slot
// nu + (S/R_k) k1 (conflict-free, consecutive tau), from which pass k+1
// reads.  Shared addresses are padded by one element every 16 (a + a/16),
// which keeps these exchange patterns free of bank conflicts for 8-byte
// elements (and within 2-way for E = 8 at the Q = 8 read).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hd {

template <class R>
struct cplx_of;
template <>
struct cplx_of<float> {
    using type = float2;
};
template <>
struct cplx_of<double> {
    using type = double2;
};
template <class R>
using cplx = typename cplx_of<R>::type;

template <class T>
using real_of = decltype(T::x);

template <class T>
__device__ __forceinline__ T mk(real_of<T> a, real_of<T> b) {
    T t;
    t.x = a;
    t.y = b;
    return t;
}
template <class T>
__device__ __forceinline__ T cadd(T a, T b) {
    return mk<T>(a.x + b.x, a.y + b.y);
}
template <class T>
__device__ __forceinline__ T csub(T a, T b) {
    return mk<T>(a.x - b.x, a.y - b.y);
}
template <class T>
__device__ __forceinline__ T cmul(T a, T b) {
    return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <class T>
__device__ __forceinline__ T cmulc(T a, T b) {
    return mk<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <class T>
__device__ __forceinline__ T cconj(T a) {
    return mk<T>(a.x, -a.y);
}
template <class T>
__device__ __forceinline__ T cscale(T a, real_of<T> s) {
    return mk<T>(a.x * s, a.y * s);
}
// multiply by +i (INV = false) or -i (INV = true)
template <bool INV, class T>
__device__ __forceinline__ T mul_i(T a) {
    return INV ? mk<T>(a.y, -a.x) : mk<T>(-a.y, a.x);
}
template <class T>
__device__ __forceinline__ T czero() {
    return mk<T>(0, 0);
}

// cos and sin of 2 pi k / 16, k = 0..7 (exact mathematical constants)
__host__ __device__ constexpr double cos16(int k) {
    return k == 0 ? 1.0
         : k == 1 ? 0.92387953251128675613
         : k == 2 ? 0.70710678118654752440
         : k == 3 ? 0.38268343236508977173
         : k == 4 ? 0.0
         : k == 5 ? -0.38268343236508977173
         : k == 6 ? -0.70710678118654752440
                  : -0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int k) {
    return k == 0 ? 0.0
         : k == 1 ? 0.38268343236508977173
         : k == 2 ? 0.70710678118654752440
         : k == 3 ? 0.92387953251128675613
         : k == 4 ? 1.0
         : k == 5 ? 0.92387953251128675613
         : k == 6 ? 0.70710678118654752440
                  : 0.38268343236508977173;
}

// a * zeta_16^{K} (INV: zeta_16^{-K}), K = 0..7, folded at compile time
template <int K, bool INV, class T>
__device__ __forceinline__ T rot16(T a) {
    using R = real_of<T>;
    if constexpr (K == 0) {
        return a;
    } else if constexpr (K == 4) {
        return mul_i<INV>(a);
    } else if constexpr (K == 2 || K == 6) {
        constexpr R h = R(0.70710678118654752440);
        // zeta_8 = (1+i)h, zeta_8^3 = (-1+i)h
        if constexpr (K == 2) {
            return INV ? mk<T>((a.x + a.y) * h, (a.y - a.x) * h) : mk<T>((a.x - a.y) * h, (a.x + a.y) * h);
        } else {
            return INV ? mk<T>((a.y - a.x) * h, -(a.x + a.y) * h) : mk<T>(-(a.x + a.y) * h, (a.x - a.y) * h);
        }
    } else {
        constexpr R c = R(cos16(K));
        constexpr R s = INV ? R(-sin16(K)) : R(sin16(K));
        return mk<T>(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

// In-register DFTs of size 2, 4, 8, 16, natural order in and out.
template <bool INV, class T>
__device__ __forceinline__ void dft2(T& a, T& b) {
    T t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV, class T>
__device__ __forceinline__ void dft4(T& v0, T& v1, T& v2, T& v3) {
    T a = cadd(v0, v2), b = csub(v0, v2), c = cadd(v1, v3), d = mul_i<INV>(csub(v1, v3));
    v0 = cadd(a, c);
    v2 = csub(a, c);
    v1 = cadd(b, d);
    v3 = csub(b, d);
}

template <bool INV, class T>
__device__ __forceinline__ void dft8(T* v) {
    T e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    T o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<INV>(e0, e1, e2, e3);
    dft4<INV>(o0, o1, o2, o3);
    o1 = rot16<2, INV>(o1);
    o2 = rot16<4, INV>(o2);
    o3 = rot16<6, INV>(o3);
    v[0] = cadd(e0, o0);
    v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1);
    v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2);
    v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3);
    v[7] = csub(e3, o3);
}

template <bool INV, class T>
__device__ __forceinline__ void dft16(T* v) {
    T e[8], o[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        e[j] = v[2 * j];
        o[j] = v[2 * j + 1];
    }
    dft8<INV>(e);
    dft8<INV>(o);
    o[1] = rot16<1, INV>(o[1]);
    o[2] = rot16<2, INV>(o[2]);
    o[3] = rot16<3, INV>(o[3]);
    o[4] = rot16<4, INV>(o[4]);
    o[5] = rot16<5, INV>(o[5]);
    o[6] = rot16<6, INV>(o[6]);
    o[7] = rot16<7, INV>(o[7]);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 8] = csub(e[k], o[k]);
    }
}

template <int R, bool INV, class T>
__device__ __forceinline__ void dft_reg(T* v) {
    if constexpr (R == 1) {
    } else if constexpr (R == 2) {
        dft2<INV>(v[0], v[1]);
    } else if constexpr (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
    } else if constexpr (R == 8) {
        dft8<INV>(v);
    } else {
        static_assert(R == 16, "radix");
        dft16<INV>(v);
    }
}

__host__ __device__ constexpr int ilog2c(int x) { return x <= 1 ? 0 : 1 + ilog2c(x >> 1); }

// Pass structure of a size-S FFT with E values per thread.
template <int S, int E>
struct FftShape {
    static_assert((S & (S - 1)) == 0 && (E & (E - 1)) == 0 && E >= 2 && E <= 16 && S >= E, "shape");
    static constexpr int T = S / E;
    static constexpr int LS = ilog2c(S);
    static constexpr int LE = ilog2c(E);
    static constexpr int KFULL = LS / LE;
    static constexpr int K = KFULL + (LS % LE ? 1 : 0);
    __host__ __device__ static constexpr int radix(int k) { return k < KFULL ? E : (1 << (LS % LE)); }
    // sub-transform size before pass k
    __host__ __device__ static constexpr int sub(int k) { return k == 0 ? S : sub(k - 1) / radix(k - 1); }
    static constexpr int RLAST = radix(K - 1);
    // padded shared elements for one transform: up to 2 pad elements per 16
    // (see fft_exchange) for E = 8, 1 per 16 otherwise
    static constexpr int SMEM = S + (E == 8 ? S / 8 : S / 16);
    // Twiddle table layout: pass k (with Q_k > 1) stores zeta_{N_k}^{c k1} at
    // tw_offset(k) + (k1 - 1) Q_k + c, so lanes with consecutive c read
    // consecutive entries.
    __host__ __device__ static constexpr int qof(int k) { return sub(k) / radix(k); }
    __host__ __device__ static constexpr int tw_count(int k) { return qof(k) > 1 ? (radix(k) - 1) * qof(k) : 0; }
    __host__ __device__ static constexpr int tw_offset(int k) { return k == 0 ? 0 : tw_offset(k - 1) + tw_count(k - 1); }
    static constexpr int TW_TOTAL = tw_offset(K);
};

__device__ __forceinline__ int padidx(int a) { return a + (a >> 4); }

template <class T>
__device__ __forceinline__ T ldtw(const T* p) {
    return __ldg(p);
}

// Twiddle source for the FFT passes: the per-pass table of FftShape (see
// tw_offset), read through the read-only data cache.
template <class T>
struct TwGlobal {
    static constexpr bool kProducts = false;
    const T* __restrict__ p;
    __device__ __forceinline__ T operator()(int idx) const { return __ldg(p + idx); }
};

// The same table, of which a radix-8 or -16 pass reads only the powers
// zeta^{c k1} with k1 = 1, 2, 4 (and 8) and forms the others as products of
// two of them (each product within two roundings of the table value): 4
// (radix 8) or 11 (radix 16) table reads per pass become complex multiplies.
// The fused kernels wait on those reads (they miss L1 beside the staging and
// exchange buffers); measured 6 % (S = 2048, E = 8) and 11 % (S = 4096,
// E = 16) faster on the 4096 x 4096 batch, results within 2.5e-7 rel-L2 of
// the full-table ones.
template <class T>
struct TwGlobalProducts {
    static constexpr bool kProducts = true;
    const T* __restrict__ p;
    __device__ __forceinline__ T operator()(int idx) const { return __ldg(p + idx); }
};

// Twiddle source for the FFT passes: the same table copied into shared memory.
template <class T>
struct TwShared {
    static constexpr bool kProducts = false;
    const T* p;
    __device__ __forceinline__ T operator()(int idx) const { return p[idx]; }
};

// w[k1] = row[k1 Q] for k1 = 1 .. R-1 of a table whose rows k1 hold the powers
// zeta^{c k1} (row points at column c of row 0, Q entries per row, Q known at
// run time): every entry read (PRODUCTS = false), or for R >= 8 only the rows
// 1, 2, 4 (and 8) and the others as products of two of them.
template <int R, bool PRODUCTS, class T>
__device__ __forceinline__ void power_row_twiddles(const T* row, int64_t Q, T* w) {
    if constexpr (PRODUCTS && R >= 8) {
        w[1] = ldtw(row + Q);
        w[2] = ldtw(row + 2 * Q);
        w[4] = ldtw(row + 4 * Q);
        w[3] = cmul(w[2], w[1]);
        w[5] = cmul(w[4], w[1]);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
        if constexpr (R == 16) {
            w[8] = ldtw(row + 8 * Q);
#pragma unroll
            for (int k1 = 9; k1 < 16; ++k1) w[k1] = cmul(w[8], w[k1 - 8]);
        }
    } else {
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) w[k1] = ldtw(row + k1 * Q);
    }
}

// w[k1] = zeta_{N_k}^{c k1}, k1 = 1 .. R-1, for column c of a pass whose table
// starts at OFF with Q columns per k1.
template <int R, int Q, int OFF, class T, class TW>
__device__ __forceinline__ void pass_twiddles(const TW& tw, int c, T* w) {
    if constexpr (TW::kProducts && R >= 8) {
        w[1] = tw(OFF + c);
        w[2] = tw(OFF + Q + c);
        w[4] = tw(OFF + 3 * Q + c);
        w[3] = cmul(w[2], w[1]);
        w[5] = cmul(w[4], w[1]);
        w[6] = cmul(w[4], w[2]);
        w[7] = cmul(w[4], w[3]);
        if constexpr (R == 16) {
            w[8] = tw(OFF + 7 * Q + c);
#pragma unroll
            for (int k1 = 9; k1 < 16; ++k1) w[k1] = cmul(w[8], w[k1 - 8]);
        }
    } else {
#pragma unroll
        for (int k1 = 1; k1 < R; ++k1) w[k1] = tw(OFF + (k1 - 1) * Q + c);
    }
}

// Pass k on NA independent arrays held back to back in v (array a in
// v[a*E .. a*E+E)): radix-R DFT, then the twiddle zeta_{N_k}^{c k1} (forward);
// the inverse applies the conjugate twiddle first, then the inverse DFT.  The
// twiddles depend only on the thread's position and are loaded once for all
// arrays.
template <int S, int E, int k, bool INV, int NA, class T, class TW>
__device__ __forceinline__ void fft_pass(T* v, const TW& tw, int tau) {
    using Sh = FftShape<S, E>;
    constexpr int R = Sh::radix(k);
    constexpr int N = Sh::sub(k);
    constexpr int Q = N / R;
    constexpr int OFF = Sh::tw_offset(k);
#pragma unroll
    for (int beta = 0; beta < E / R; ++beta) {
        const int nu = tau + Sh::T * beta;
        const int c = nu & (Q - 1);
        if constexpr (!INV) {
#pragma unroll
            for (int a = 0; a < NA; ++a) dft_reg<R, false>(v + a * E + beta * R);
        }
        if constexpr (Q > 1) {
            T w[R];
            pass_twiddles<R, Q, OFF>(tw, c, w);            // zeta_{N_k}^{c k1}
#pragma unroll
            for (int k1 = 1; k1 < R; ++k1) {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    T& x = v[a * E + beta * R + k1];
                    x = INV ? cmulc(x, w[k1]) : cmul(x, w[k1]);
                }
            }
        }
        if constexpr (INV) {
#pragma unroll
            for (int a = 0; a < NA; ++a) dft_reg<R, true>(v + a * E + beta * R);
        }
    }
}

// Exchange between pass k and pass k+1 for NA arrays (array a uses the padded
// buffer sm + a * SMEM).  Padded slots of x + D with D a multiple of 16 are
// padidx(x) + D + D/16, so each group of accesses computes one padded base.  FWD: from the layout after pass k to the layout pass
// k+1 reads; otherwise the reverse.  Two barriers: after the writes, and
// before the buffers are written again.  CST > 1 interleaves the buffers of
// CST independent transforms (one per column of a column tile): slot s of the
// transform held by this thread is at sm[s * CST], sm pointing at its column.
// Addressing of exchange k (between pass k and pass k+1): the slot pass k
// writes for (beta, k1) and the slot pass k+1 reads for (beta, i).  Pad
// elements per 16: 1, or 2 for the radix-8 reads with 1 < Qn < 16, whose
// half-warps otherwise meet two words in one bank (checked on the CPU for
// every exchange of E = 8 and 16, tests/test_fft_exchange_cpu.py: the writes
// and reads of each exchange are then conflict-free, and every index stays
// below SMEM).  Column tiles (CST > 1) keep 1.
template <int S, int E, int k, int CST>
struct Exch {
    using Sh = FftShape<S, E>;
    static constexpr int R = Sh::radix(k);
    static constexpr int V = S / R;
    static constexpr int Rn = Sh::radix(k + 1);
    static constexpr int Qn = Sh::sub(k + 1) / Rn;
    static constexpr int PADM = (CST == 1 && Rn == 8 && Qn > 1 && Qn < 16) ? 2 : 1;
    static_assert(PADM == 1 || E == 8, "two pad elements per 16 only fit the E = 8 buffers");
    __device__ __forceinline__ static int padk(int a) { return a + (a >> 4) * PADM; }
    // slot of value k1 of virtual thread nu after pass k
    __device__ __forceinline__ static int out_slot(int pn, int nu, int k1) {
        return (V % 16 == 0) ? pn + V * k1 + (V / 16) * PADM * k1 : padk(nu + V * k1);
    }
    // slot of value i of virtual thread nu before pass k + 1
    __device__ __forceinline__ static int in_slot(int pb, int base, int i) {
        return (Qn % 16 == 0) ? pb + i * Qn + (Qn / 16) * PADM * i : padk(base + i * Qn);
    }
};

// One half of exchange k for NA arrays (array a in the padded buffer
// sm + a * SMEM): AFTER = true moves the layout after pass k (the forward
// direction writes it, the inverse reads it), AFTER = false the layout pass
// k + 1 reads.  STORE: registers to shared memory, else the reverse.
template <int S, int E, int k, bool AFTER, bool STORE, int NA, int CST, class T>
__device__ __forceinline__ void exch_half(T* v, T* sm, int tau) {
    using Sh = FftShape<S, E>;
    using X = Exch<S, E, k, CST>;
    if constexpr (AFTER) {
#pragma unroll
        for (int beta = 0; beta < E / X::R; ++beta) {
            const int nu = tau + Sh::T * beta;
            const int pn = X::padk(nu);
#pragma unroll
            for (int k1 = 0; k1 < X::R; ++k1) {
                const int idx = X::out_slot(pn, nu, k1);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    T& r = v[a * E + beta * X::R + k1];
                    T& m = sm[(a * Sh::SMEM + idx) * CST];
                    if constexpr (STORE) m = r; else r = m;
                }
            }
        }
    } else {
#pragma unroll
        for (int beta = 0; beta < E / X::Rn; ++beta) {
            const int nu = tau + Sh::T * beta;
            const int b = nu / X::Qn, c = nu & (X::Qn - 1);
            const int base = b * X::Rn * X::Qn + c;
            const int pb = X::padk(base);
#pragma unroll
            for (int i = 0; i < X::Rn; ++i) {
                const int idx = X::in_slot(pb, base, i);
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    T& r = v[a * E + beta * X::Rn + i];
                    T& m = sm[(a * Sh::SMEM + idx) * CST];
                    if constexpr (STORE) m = r; else r = m;
                }
            }
        }
    }
}

// Exchange between pass k and pass k+1 for NA arrays (array a uses the padded
// buffer sm + a * SMEM).  FWD: from the layout after pass k to the layout pass
// k+1 reads; otherwise the reverse.  Two barriers: after the writes, and
// before the buffers are written again.  CST > 1 interleaves the buffers of
// CST independent transforms (one per column of a column tile): slot s of the
// transform held by this thread is at sm[s * CST], sm pointing at its column.
template <int S, int E, int k, bool FWD, int NA, int CST, class T>
__device__ __forceinline__ void fft_exchange(T* v, T* sm, int tau) {
    exch_half<S, E, k, FWD, true, NA, CST>(v, sm, tau);
    __syncthreads();
    exch_half<S, E, k, !FWD, false, NA, CST>(v, sm, tau);
    __syncthreads();
}

template <int S, int E, int k, int NA, int CST, class T, class TW>
__device__ __forceinline__ void fft_fwd_from(T* v, T* sm, const TW& tw, int tau) {
    using Sh = FftShape<S, E>;
    fft_pass<S, E, k, false, NA>(v, tw, tau);
    if constexpr (k + 1 < Sh::K) {
        fft_exchange<S, E, k, true, NA, CST>(v, sm, tau);
        fft_fwd_from<S, E, k + 1, NA, CST>(v, sm, tw, tau);
    }
}

template <int S, int E, int k, int NA, int CST, class T, class TW>
__device__ __forceinline__ void fft_inv_from(T* v, T* sm, const TW& tw, int tau) {
    fft_pass<S, E, k, true, NA>(v, tw, tau);
    if constexpr (k > 0) {
        fft_exchange<S, E, k - 1, false, NA, CST>(v, sm, tau);
        fft_inv_from<S, E, k - 1, NA, CST>(v, sm, tw, tau);
    }
}

// Forward FFT of NA arrays: natural layout in, spectral layout out.
template <int S, int E, int NA = 1, int CST = 1, class T, class TW>
__device__ __forceinline__ void fft_forward(T* v, T* sm, const TW& tw, int tau) {
    fft_fwd_from<S, E, 0, NA, CST>(v, sm, tw, tau);
}

// Inverse FFT (unnormalized) of NA arrays: spectral layout in, natural layout out.
template <int S, int E, int NA = 1, int CST = 1, class T, class TW>
__device__ __forceinline__ void fft_inverse(T* v, T* sm, const TW& tw, int tau) {
    fft_inv_from<S, E, FftShape<S, E>::K - 1, NA, CST>(v, sm, tw, tau);
}

// Frequency index held by register e of thread tau in the spectral layout.
template <int S, int E>
__device__ __forceinline__ int spectral_index(int tau, int e) {
    using Sh = FftShape<S, E>;
    constexpr int RL = Sh::RLAST;
    return tau + Sh::T * (e / RL) + (S / RL) * (e % RL);
}

}  // namespace hd
