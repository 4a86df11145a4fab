// Lagrange interpolation weights and their derivatives on the device
// (Sec. 3.2): w_j(t) = prod_{l != j} (t - l) / (j - l) for the nodes
// j = 0..p of a stencil, t the local coordinate in grid steps.
#pragma once
#include "pim_internal.cuh"

namespace pim_k {

// Lagrange weights of compile-time degree P (prefix/suffix products times
// the constant inverse denominators).
template <typename T, int P>
__device__ __forceinline__ void lagrange_w(T t, T* w) {
    T pre[P + 1], suf[P + 1];
    pre[0] = T(1);
#pragma unroll
    for (int j = 1; j <= P; ++j) pre[j] = pre[j - 1] * (t - T(j - 1));
    suf[P] = T(1);
#pragma unroll
    for (int j = P - 1; j >= 0; --j) suf[j] = suf[j + 1] * (t - T(j + 1));
#pragma unroll
    for (int j = 0; j <= P; ++j) {
        double den = 1.0;
        for (int l = 0; l <= P; ++l)
            if (l != j) den *= (double)(j - l);
        w[j] = pre[j] * suf[j] * T(1.0 / den);
    }
}

// Inverse Lagrange denominator 1 / prod_{l != j, l <= p} (j - l) of node j
// at degree p (Sec. 3.2), evaluated at compile time.
constexpr double lag_inv_den(int p, int j) {
    double den = 1.0;
    for (int l = 0; l <= p; ++l)
        if (l != j) den *= (double)(j - l);
    return 1.0 / den;
}
struct LagInv {
    double v[PIM_MAX_P + 1][PIM_MAX_P + 1];
};
constexpr LagInv make_lag_inv() {
    LagInv r{};
    for (int p = 0; p <= PIM_MAX_P; ++p)
        for (int j = 0; j <= p; ++j) r.v[p][j] = lag_inv_den(p, j);
    return r;
}
__constant__ LagInv c_lag_inv = make_lag_inv();

// One Lagrange weight w_j(t) of compile-time degree P for a runtime node j.
template <typename T, int P>
__device__ __forceinline__ T lag1(T t, int j) {
    T r = T(1), c = T(lag_inv_den(P, 0));
#pragma unroll
    for (int l = 0; l <= P; ++l) {
        r *= (l == j) ? T(1) : (t - T(l));
        if (l > 0) c = (l == j) ? T(lag_inv_den(P, l)) : c;
    }
    return r * c;
}

// One Lagrange weight w_j(t) of runtime degree p <= PIM_MAX_P.
template <typename T>
__device__ __forceinline__ T lag1_rt(int p, T t, int j) {
    T r = T(1);
#pragma unroll
    for (int l = 0; l <= PIM_MAX_P; ++l) r *= (l == j || l > p) ? T(1) : (t - T(l));
    return r * T(c_lag_inv.v[p][j]);
}

// Lagrange weights of runtime degree p <= PIM_MAX_P without divisions
// (prefix/suffix products times the tabulated inverse denominators).
template <typename T>
__device__ __forceinline__ void lagrange_w_rt(int p, T t, T* w) {
    T pre[PIM_MAX_P + 1], suf[PIM_MAX_P + 1];
    pre[0] = T(1);
#pragma unroll
    for (int j = 1; j <= PIM_MAX_P; ++j) pre[j] = pre[j - 1] * (t - T(j - 1));
    suf[PIM_MAX_P] = T(1);
#pragma unroll
    for (int j = PIM_MAX_P - 1; j >= 0; --j) suf[j] = (j + 1 <= p) ? suf[j + 1] * (t - T(j + 1)) : T(1);
#pragma unroll
    for (int j = 0; j <= PIM_MAX_P; ++j) w[j] = j <= p ? pre[j] * suf[j] * T(c_lag_inv.v[p][j]) : T(0);
}

// Derivatives of the Lagrange basis of degree P (product rule).
template <typename T, int P>
__device__ __forceinline__ void lagrange_dw(T t, T* dw) {
#pragma unroll
    for (int j = 0; j <= P; ++j) {
        double den = 1.0;
        for (int l = 0; l <= P; ++l)
            if (l != j) den *= (double)(j - l);
        T s = T(0);
#pragma unroll
        for (int k = 0; k <= P; ++k) {
            if (k == j) continue;
            T pr = T(1);
#pragma unroll
            for (int l = 0; l <= P; ++l)
                if (l != j && l != k) pr *= (t - T(l));
            s += pr;
        }
        dw[j] = s * T(1.0 / den);
    }
}

template <typename T>
__device__ __forceinline__ void lagrange_dw_rt(int p, T t, T* dw) {
#pragma unroll
    for (int j = 0; j <= PIM_MAX_P; ++j) {
        T den = T(1), s = T(0);
#pragma unroll
        for (int l = 0; l <= PIM_MAX_P; ++l)
            if (l != j && l <= p) den *= T(j - l);
#pragma unroll
        for (int k = 0; k <= PIM_MAX_P; ++k) {
            if (k == j || k > p) continue;
            T pr = T(1);
#pragma unroll
            for (int l = 0; l <= PIM_MAX_P; ++l)
                if (l != j && l != k && l <= p) pr *= (t - T(l));
            s += pr;
        }
        dw[j] = j <= p ? s / den : T(0);
    }
}

// Weights and their t-derivatives together, O(P) per node: prefix and suffix
// products of (t - l) and, by the product rule, their derivatives.
template <typename T, int P>
__device__ __forceinline__ void lagrange_wdw(T t, T* w, T* dw) {
    T pre[P + 1], dpre[P + 1], suf[P + 1], dsuf[P + 1];
    pre[0] = T(1);
    dpre[0] = T(0);
#pragma unroll
    for (int j = 1; j <= P; ++j) {
        pre[j] = pre[j - 1] * (t - T(j - 1));
        dpre[j] = dpre[j - 1] * (t - T(j - 1)) + pre[j - 1];
    }
    suf[P] = T(1);
    dsuf[P] = T(0);
#pragma unroll
    for (int j = P - 1; j >= 0; --j) {
        suf[j] = suf[j + 1] * (t - T(j + 1));
        dsuf[j] = dsuf[j + 1] * (t - T(j + 1)) + suf[j + 1];
    }
#pragma unroll
    for (int j = 0; j <= P; ++j) {
        const T c = T(lag_inv_den(P, j));
        w[j] = pre[j] * suf[j] * c;
        dw[j] = (dpre[j] * suf[j] + pre[j] * dsuf[j]) * c;
    }
}

// The same for a runtime degree p <= PIM_MAX_P (entries above p are zero).
template <typename T>
__device__ __forceinline__ void lagrange_wdw_rt(int p, T t, T* w, T* dw) {
    T pre[PIM_MAX_P + 1], dpre[PIM_MAX_P + 1], suf[PIM_MAX_P + 1], dsuf[PIM_MAX_P + 1];
    pre[0] = T(1);
    dpre[0] = T(0);
#pragma unroll
    for (int j = 1; j <= PIM_MAX_P; ++j) {
        pre[j] = pre[j - 1] * (t - T(j - 1));
        dpre[j] = dpre[j - 1] * (t - T(j - 1)) + pre[j - 1];
    }
    suf[PIM_MAX_P] = T(1);
    dsuf[PIM_MAX_P] = T(0);
#pragma unroll
    for (int j = PIM_MAX_P - 1; j >= 0; --j) {
        const bool in = j + 1 <= p;
        suf[j] = in ? suf[j + 1] * (t - T(j + 1)) : T(1);
        dsuf[j] = in ? dsuf[j + 1] * (t - T(j + 1)) + suf[j + 1] : T(0);
    }
#pragma unroll
    for (int j = 0; j <= PIM_MAX_P; ++j) {
        const T c = j <= p ? T(c_lag_inv.v[p][j]) : T(0);
        w[j] = pre[j] * suf[j] * c;
        dw[j] = (dpre[j] * suf[j] + pre[j] * dsuf[j]) * c;
    }
}

}  // namespace pim_k
