// regfft.cuh - FP32 DFTs of compile-time length held in registers, and the compile-time
// twiddle constants they use (the building blocks of the four-step transforms of the column
// and row kernels; FluTAS Sec. 3.3.1, the transforms along x, y and z).
#pragma once
#include <type_traits>
#include <utility>

#include <cuda_runtime.h>

namespace {

// ------------------------------------------------ compile-time twiddle constants
constexpr double kPi = 3.14159265358979323846264338327950288;

// sin x and cos x for |x| <= pi/4 from their Taylor series (terms to x^23, the remainder
// is below 1e-30 there).
__host__ __device__ constexpr double taylor_sin(double x) {
    double x2 = x * x, t = x, s = x;
    for (int i = 1; i <= 11; ++i) {
        t *= -x2 / (double)((2 * i) * (2 * i + 1));
        s += t;
    }
    return s;
}
__host__ __device__ constexpr double taylor_cos(double x) {
    double x2 = x * x, t = 1.0, s = 1.0;
    for (int i = 1; i <= 11; ++i) {
        t *= -x2 / (double)((2 * i - 1) * (2 * i));
        s += t;
    }
    return s;
}
// cos(2 pi m / n) or sin(2 pi m / n): the angle is split exactly, in integers, into q quarter
// turns and a fraction e/n of a quarter turn; the fraction's sine and cosine come from the
// series at an argument of at most pi/4 (the complement is used above pi/4).
__host__ __device__ constexpr double cs2pi(long long m, long long n, bool want_sin) {
    const long long r = ((m % n) + n) % n;
    const long long q = (4 * r) / n, e = 4 * r - q * n;
    double ce = 0.0, se = 0.0;
    if (2 * e <= n) {
        const double x = (double)e / (double)n * (kPi / 2);
        ce = taylor_cos(x);
        se = taylor_sin(x);
    } else {
        const double x = (double)(n - e) / (double)n * (kPi / 2);
        ce = taylor_sin(x);
        se = taylor_cos(x);
    }
    double c = ce, s = se;
    if (q == 1) { c = -se; s = ce; }
    else if (q == 2) { c = -ce; s = -se; }
    else if (q == 3) { c = se; s = -ce; }
    return want_sin ? s : c;
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = 0 .. N-1, so that every index
// inside f is a constant expression.
template <typename F, int... I>
__device__ __forceinline__ void sfor_seq(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void sfor(F&& f) {
    sfor_seq(f, std::make_integer_sequence<int, N>{});
}

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// a W_R^M (forward) or a W_R^-M (inverse) for a compile-time M: quarter turns by swaps and
// signs, every other angle by a product with constants.
template <int R, int M, bool INV>
__device__ __forceinline__ float2 ktw(float2 a) {
    constexpr int m = ((M % R) + R) % R;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (2 * m == R) {
        return make_float2(-a.x, -a.y);
    } else if constexpr (4 * m == R) {                 // W^(R/4) = -i
        return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
    } else if constexpr (4 * m == 3 * R) {             // W^(3R/4) = +i
        return INV ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
    } else {
        constexpr float c = (float)cs2pi(m, R, false);
        constexpr float s = (float)cs2pi(m, R, true);
        if (INV) return make_float2(fmaf(a.x, c, -a.y * s), fmaf(a.y, c, a.x * s));
        return make_float2(fmaf(a.x, c, a.y * s), fmaf(a.y, c, -a.x * s));
    }
}

// 1/x by the hardware reciprocal approximation (relative error about 2^-23, one rounding of
// the FP32 transforms' size; the FP64 defect correction removes it like any FP32 rounding).
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// a w (forward) or a conj(w) (inverse) for a twiddle w from a table.
template <bool INV>
__device__ __forceinline__ float2 tmul(float2 a, float2 w) {
    if (INV) return make_float2(fmaf(a.x, w.x, a.y * w.y), fmaf(a.y, w.x, -a.x * w.y));
    return make_float2(fmaf(a.x, w.x, -a.y * w.y), fmaf(a.x, w.y, a.y * w.x));
}

// ------------------------------------------------ DFTs of compile-time length in registers
// X[k] = sum_n v[n] W_R^(+-nk), natural order in and out.
template <int R, bool INV> struct RegDft;

template <bool INV> struct RegDft<2, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float2 a = v[0];
        v[0] = c_add(a, v[1]);
        v[1] = c_sub(a, v[1]);
    }
};

template <bool INV> struct RegDft<4, INV> {
    __device__ __forceinline__ static void run(float2* v) {
        const float2 s02 = c_add(v[0], v[2]), d02 = c_sub(v[0], v[2]), s13 = c_add(v[1], v[3]);
        const float2 e = c_sub(v[1], v[3]);
        const float2 d13 = INV ? make_float2(-e.y, e.x) : make_float2(e.y, -e.x);   // (x1 - x3) W_4^(+-1)
        v[0] = c_add(s02, s13);
        v[2] = c_sub(s02, s13);
        v[1] = c_add(d02, d13);
        v[3] = c_sub(d02, d13);
    }
};

// R = A Bq by the same four steps as the column transform, all indices constant.
template <int A, int Bq, bool INV>
__device__ __forceinline__ void reg_four_step(float2* v) {
    constexpr int R = A * Bq;
    float2 y[R];
    sfor<Bq>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        float2 sub[A];
        sfor<A>([&](auto n1c) { sub[decltype(n1c)::value] = v[Bq * decltype(n1c)::value + n2]; });
        RegDft<A, INV>::run(sub);
        sfor<A>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            y[k1 * Bq + n2] = ktw<R, n2 * k1, INV>(sub[k1]);
        });
    });
    sfor<A>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        float2 sub[Bq];
        sfor<Bq>([&](auto n2c) { sub[decltype(n2c)::value] = y[k1 * Bq + decltype(n2c)::value]; });
        RegDft<Bq, INV>::run(sub);
        sfor<Bq>([&](auto k2c) { v[k1 + A * decltype(k2c)::value] = sub[decltype(k2c)::value]; });
    });
}

template <bool INV> struct RegDft<8, INV> {
    __device__ __forceinline__ static void run(float2* v) { reg_four_step<4, 2, INV>(v); }
};
template <bool INV> struct RegDft<16, INV> {
    __device__ __forceinline__ static void run(float2* v) { reg_four_step<4, 4, INV>(v); }
};
template <bool INV> struct RegDft<32, INV> {
    __device__ __forceinline__ static void run(float2* v) { reg_four_step<8, 4, INV>(v); }
};

}  // namespace
