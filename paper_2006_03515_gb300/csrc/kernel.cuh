// The photoionization kernel on the device (Eqs. (integral) and (gfun) of the paper):
//   K(R) = (exp(-aR) - exp(-bR)) / (4 pi R^3 ln(b/a)),  a = chi_min p_O2, b = chi_max p_O2.
// Both forms write the difference as exp(-aR) * (1 - exp(-(b-a)R)) so that it keeps
// its relative precision when (b-a)R is small (low pressure).
#pragma once
#include <cuda_runtime.h>

namespace kifmm {

struct KParams {
    double a, b, bma, norm;   // norm = 1 / (4 pi ln(b/a))
    float a_l2e, bma_l2e, bma_f, norm_f;   // FP32 forms: a*log2(e), (b-a)*log2(e), b-a, norm
    float b_l2e;                           // b*log2(e)
    float r_series;                        // 0.5 / (b - a): below it 1 - e^{-(b-a)R} uses the series
    // comparison kernels (kind != 0): K(R) = sum_j w_j exp(-kap_j R) / R^alpha
    int kind = 0, alpha = 0, nterm = 0;
    double w[3] = {0, 0, 0}, kap[3] = {0, 0, 0};
};

inline KParams make_kparams(double a, double b) {
    KParams k;
    k.a = a;
    k.b = b;
    k.bma = b - a;
    k.norm = 1.0 / (4.0 * 3.14159265358979323846 * log(b / a));
    const double l2e = 1.4426950408889634074;
    k.a_l2e = (float)(a * l2e);
    k.bma_l2e = (float)((b - a) * l2e);
    k.bma_f = (float)(b - a);
    k.norm_f = (float)k.norm;
    k.b_l2e = (float)(b * l2e);
    k.r_series = (float)(0.5 / (b - a));
    return k;
}

// The comparison models' kernels through the same sum, at p_O2 = a / chi_min (chi_min = 0.035):
// kind 1, Sec. 2.2, Eq. (gexp), Table Helcoeff: sum_j C_j p_O2^2 exp(-lambda_j p_O2 R) / (4 pi R)
// (the modified Helmholtz equations' free-space Green's functions); kind 2, Sec. 2.3,
// Eq. (rtetoint), Table threegroupcoeff: sum_j A_j p_O2 exp(-lambda_j p_O2 R) / (4 pi R^2).
inline KParams make_kparams_kind(int kind, double a, double b) {
    KParams k = make_kparams(a, b);
    if (kind != 1 && kind != 2) return k;
    const double p = a / 0.035, pi4 = 4.0 * 3.14159265358979323846;
    const double hel[3][2] = {{1.986e-4, 0.0553}, {0.0051, 0.1460}, {0.4886, 0.89}};
    const double grp[3][2] = {{0.0067, 0.0447}, {0.0346, 0.1121}, {0.3059, 0.5994}};
    k.kind = kind;
    k.alpha = kind;
    k.nterm = 3;
    for (int j = 0; j < 3; ++j) {
        k.w[j] = kind == 1 ? hel[j][0] * p * p / pi4 : grp[j][0] * p / pi4;
        k.kap[j] = (kind == 1 ? hel[j][1] : grp[j][1]) * p;
    }
    return k;
}

// FP64: CUDA's exp / expm1.
__device__ __forceinline__ double kern_f64(double R, const KParams& k) {
    if (k.kind) {
        double s = 0.0;
        for (int j = 0; j < k.nterm; ++j) s += k.w[j] * exp(-k.kap[j] * R);
        return k.alpha == 1 ? s / R : s / (R * R);
    }
    return -exp(-k.a * R) * expm1(-k.bma * R) * k.norm / (R * R * R);
}

// int_0^R K(r) r^2 dr (the flux of the kernel's mass through a sphere of radius R over 4 pi),
// for the self-cell integrals; kind 0 through E1 (e1 the exponential integral)
template <class E1>
__device__ __forceinline__ double kern_mass(double R, const KParams& k, E1 e1) {
    if (k.kind) {
        double s = 0.0;
        for (int j = 0; j < k.nterm; ++j) {
            const double x = k.kap[j] * R;
            s += k.alpha == 1 ? k.w[j] * (-expm1(-x) - x * exp(-x)) / (k.kap[j] * k.kap[j])
                              : k.w[j] * (-expm1(-x)) / k.kap[j];
        }
        return s;
    }
    const double lba = log(k.b / k.a);
    return (lba + e1(k.b * R) - e1(k.a * R)) * k.norm;
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1 - exp(-x) for x >= 0 in FP32. For x < 0.5 the Maclaurin series of 1 - e^{-x},
// x (1 - x/2 (1 - x/3 (1 - ... (1 - x/10)))), truncated after the x^10 term
// (relative truncation error below x^10/11! < 3e-11 for x < 0.5); otherwise
// 1 - 2^{-x log2 e}, where the subtraction loses at most a factor 1/(1 - e^{-0.5}) = 2.5.
__device__ __forceinline__ float one_minus_exp_neg(float x, float x_l2e) {
    if (x < 0.5f) {
        float t = 1.0f - x * (1.0f / 10.0f);
        t = 1.0f - x * (1.0f / 9.0f) * t;
        t = 1.0f - x * (1.0f / 8.0f) * t;
        t = 1.0f - x * (1.0f / 7.0f) * t;
        t = 1.0f - x * (1.0f / 6.0f) * t;
        t = 1.0f - x * (1.0f / 5.0f) * t;
        t = 1.0f - x * (1.0f / 4.0f) * t;
        t = 1.0f - x * (1.0f / 3.0f) * t;
        t = 1.0f - x * 0.5f * t;
        return x * t;
    }
    return 1.0f - ex2_approx(-x_l2e);
}

// FP32 kernel from the squared distance r2 > 0 (box-local coordinates); the paper's kernel
// only (the comparison kernels run in the FP64 form).
__device__ __forceinline__ float kern_f32(float r2, const KParams& k) {
    const float rinv = rsqrt_approx(r2);
    const float R = r2 * rinv;
    const float ea = ex2_approx(-k.a_l2e * R);
    const float m1 = one_minus_exp_neg(k.bma_f * R, k.bma_l2e * R);
    return ea * m1 * k.norm_f * (rinv * rinv * rinv);
}

// e^{-aR} - e^{-bR} in FP32. For (b-a)R >= 0.5 the plain difference of the two
// exponentials (relative error amplified at most 1/(1 - e^{-0.5}) = 2.5x); below, the
// factored form e^{-aR} (1 - e^{-(b-a)R}) with the series for the bracket.
__device__ __forceinline__ float exp_diff_f32(float R, const KParams& k) {
    if (R < k.r_series) return ex2_approx(-k.a_l2e * R) * one_minus_exp_neg(k.bma_f * R, k.bma_l2e * R);
    return ex2_approx(-k.a_l2e * R) - ex2_approx(-k.b_l2e * R);
}

// Kahan-compensated FP32 accumulator
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        float y = v - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace kifmm
