// The gather of the apply (Sec. 3.3 steps 3-4): the fused near-grid
// interpolation and CSR near-pair correction, one warp per point, with its
// launch-shape variants.
#pragma once
#include "lagrange.cuh"
#include "pim_internal.cuh"

namespace pim_k {

struct GatherArgs {
    int n[3], nf[3], pf;
    long long N;
    int nrhs, r;
    int cmode, adj, has_far, real_out, sorted_out, self_img;
    const int* perm;
    const uint32_t* ns;
    const float* nt;
    const double* ntd;
    const uint32_t* fst;   // far stencils of the grid gathered from
    const float* ft;
    const double* ftd;
    int toff;
    const int64_t* row_ptr;
    const uint32_t* col;
    const double2* val;
    const float4* valdf;
    const float2* valf;
    const uint32_t* valt;
    const int* nbig;
    const double2* phase;
    const float4* phasedf;
};

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
    const float s = hi + b;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (b - bb);
    hi = s;
}

// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Double-float complex numbers are float4 (re hi, re lo, im hi, im lo).
// (rh + rl) + j (ih + il) += d x for a double-float d and an FP32 x, with the
// four leading products split exactly by fma and the rest in FP32.
__device__ __forceinline__ void df_cmac(float& rh, float& rl, float& ih, float& il, const float4 d, float xr,
                                        float xi) {
    const float p1 = d.x * xr, e1 = fmaf(d.x, xr, -p1);
    const float p2 = d.z * xi, e2 = fmaf(d.z, xi, -p2);
    const float p3 = d.x * xi, e3 = fmaf(d.x, xi, -p3);
    const float p4 = d.z * xr, e4 = fmaf(d.z, xr, -p4);
    two_sum_acc(rh, rl, p1);
    two_sum_acc(rh, rl, -p2);
    two_sum_acc(ih, il, p3);
    two_sum_acc(ih, il, p4);
    rl += (e1 - e2) + (d.y * xr - d.w * xi);
    il += (e3 + e4) + (d.y * xi + d.w * xr);
}

// p d for double-float p and d (the image phase times a correction value),
// rounded back to a normalised double-float pair per component.
__device__ __forceinline__ float4 df_cmul(const float4 p, const float4 d) {
    float s, e;
    float4 r;
    const float p1 = p.x * d.x, e1 = fmaf(p.x, d.x, -p1);
    const float p2 = p.z * d.z, e2 = fmaf(p.z, d.z, -p2);
    two_sum(p1, -p2, s, e);
    two_sum(s, e + (e1 - e2) + (fmaf(p.x, d.y, p.y * d.x) - fmaf(p.z, d.w, p.w * d.z)), r.x, r.y);
    const float p3 = p.x * d.z, e3 = fmaf(p.x, d.z, -p3);
    const float p4 = p.z * d.x, e4 = fmaf(p.z, d.x, -p4);
    two_sum(p3, p4, s, e);
    two_sum(s, e + (e3 + e4) + (fmaf(p.x, d.w, p.y * d.z) + fmaf(p.z, d.y, p.w * d.x)), r.z, r.w);
    return r;
}

// A compact value (FP32 head h, bf16 tails of re and im in t) as a
// double-float complex: the tails are the high halves of FP32 words.
__device__ __forceinline__ float4 compact_value(float2 h, uint32_t t) {
    return make_float4(h.x, __uint_as_float(t << 16), h.y, __uint_as_float(t & 0xffff0000u));
}

// sum of a double-float over the warp (lane 0 holds the result)
__device__ __forceinline__ void df_warp_sum(float& h, float& l) {
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        float s, e;
        two_sum(h, oh, s, e);
        h = s;
        l += ol + e;
    }
}

// Near-pair correction of one row, all lanes of the warp: entry q = lane,
// lane + 32, ... of [0, len).  Full trips take UNR entries per lane with every
// column and value load issued before the dependent source loads and no
// bounds tests; the tail takes one entry per lane.  load(q) reads the value
// of entry q; body(c, d, x) gets the column word, the value and the source q_n.
template <int UNR, typename C, typename L, typename F>
__device__ __forceinline__ void corr_row(int lane, int len, const uint32_t* __restrict__ colr, L&& load,
                                         const C* __restrict__ qs, F&& body) {
    using V = decltype(load(0));
    int q = lane;
    for (; q + 32 * (UNR - 1) < len; q += 32 * UNR) {
        uint32_t c[UNR];
        V d[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
            c[u] = __ldcs(colr + q + 32 * u);
            d[u] = load(q + 32 * u);
        }
        C x[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u) x[u] = qs[c[u] & PIM_COL_MASK];
#pragma unroll
        for (int u = 0; u < UNR; ++u) body(c[u], d[u], x[u]);
    }
    for (; q < len; q += 32) {
        const uint32_t c = __ldcs(colr + q);
        const V d = load(q);
        body(c, d, qs[c & PIM_COL_MASK]);
    }
}

// Near gather (Sec. 3.3 step 3) of point m, this lane's share: lane (jy, jz)
// takes one x-row of the stencil.
template <typename T, int P>
__device__ __forceinline__ cplx<T> near_part(const GatherArgs& a, long long m, int lane, const cplx<T>* __restrict__ U) {
    constexpr int NP = P + 1;
    cplx<T> acc = mk<T>(T(0), T(0));
    if (lane < NP * NP) {
        const int jy = lane % NP, jz = lane / NP;
        int s[3];
        unpack3(a.ns[m], s[0], s[1], s[2]);
        T t[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) t[d] = sizeof(T) == 8 ? (T)a.ntd[3 * m + d] : (T)a.nt[3 * m + d];
        const T wyz = lag1<T, P>(t[1], jy) * lag1<T, P>(t[2], jz);
        T wx[NP];
        lagrange_w<T, P>(t[0], wx);
        const cplx<T>* row = U + ((long long)(s[2] + jz) * a.n[1] + (s[1] + jy)) * a.n[0] + s[0];
        cplx<T> r = mk<T>(T(0), T(0));
#pragma unroll
        for (int jx = 0; jx < NP; ++jx) {
            const cplx<T> v = row[jx];
            r.x += wx[jx] * v.x;
            r.y += wx[jx] * v.y;
        }
        acc.x = wyz * r.x;
        acc.y = wyz * r.y;
    }
    return acc;
}

// One warp per sorted point: near gather (Sec. 3.3 step 3) and near-pair
// correction (step 4, Eq. er), summed and written in the caller's order (the
// far part is added by far_add_kernel).  In the gather lane (jy, jz) takes one
// x-row of the stencil.
template <typename T, int P, int CM, int UNR, int MINB>
__global__ void __launch_bounds__(256, MINB) gather_kernel(GatherArgs a, const cplx<T>* __restrict__ U,
                                                     const cplx<T>* __restrict__ qs, void* out) {
    const int lane = threadIdx.x & 31;
    const long long m = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (m >= a.N) return;
    cplx<T> acc = near_part<T, P>(a, m, lane, U);
    // near-pair correction: exp(-j k0.(i o L)) d q_n (forward) or
    // exp(-j k0.(i o L)) conj(d) v_n (adjoint).  The adjoint is summed as the
    // conjugate of sum conj(phase) d conj(v_n), so that the values are used
    // as stored.
    const long long r0 = CM < 0 ? 0 : a.row_ptr[m];
    const int len = CM < 0 ? 0 : (int)(a.row_ptr[m + 1] - r0);
    const uint32_t* colr = a.col + r0;
    const float fs = a.adj ? -1.f : 1.f;
    double2 accd = make_double2(0.0, 0.0);
    float rh = 0.f, rl = 0.f, ih = 0.f, il = 0.f;
    if (CM == PIM_CORR_FP64) {
        const double2* vr = a.val + r0;
        corr_row<UNR>(lane, len, colr, [=](int e) { return __ldcs(vr + e); }, qs,
                      [&](uint32_t c, const double2& d, const cplx<T>& x) {
            const double xr = (double)x.x, xi = (double)fs * (double)x.y;
            double2 t = make_double2(d.x * xr - d.y * xi, d.x * xi + d.y * xr);
            const int ii = (int)(c >> PIM_COL_BITS);
            if (ii != a.self_img) {
                const double2 ph = a.phase[ii];
                t = cmul(make_double2(ph.x, (double)fs * ph.y), t);
            }
            accd = cadd(accd, t);
        });
    } else if (corr_df(CM)) {
        // FP32 arithmetic throughout: values of other images are multiplied by
        // their phase in double-float, every entry is added by df_cmac and the
        // warp sum is double-float too
        auto body = [&](uint32_t c, const float4& d, const cplx<T>& x) {
            const int ii = (int)(c >> PIM_COL_BITS);
            float4 v = d;
            if (ii != a.self_img) {
                float4 ph = a.phasedf[ii];
                ph.z *= fs;
                ph.w *= fs;
                v = df_cmul(ph, v);
            }
            df_cmac(rh, rl, ih, il, v, (float)x.x, fs * (float)x.y);
        };
        if (CM == PIM_CORR_COMPACT) {
            // the row's large entries (double-float), then its small ones
            // (complex64 values, FP32 sums folded in once per lane)
            const int nb = a.nbig[m];
            const float2* hr = a.valf + r0;
            const uint32_t* tr = a.valt + r0;
            corr_row<UNR>(lane, nb, colr, [=](int e) { return compact_value(__ldcs(hr + e), __ldcs(tr + e)); }, qs,
                          body);
            float sr = 0.f, si = 0.f;
            corr_row<UNR>(lane, len - nb, colr + nb, [=](int e) { return __ldcs(hr + nb + e); }, qs,
                          [&](uint32_t c, const float2& d, const cplx<T>& x) {
                              const float xr = (float)x.x, xi = fs * (float)x.y;
                              float2 t = make_float2(d.x * xr - d.y * xi, d.x * xi + d.y * xr);
                              const int ii = (int)(c >> PIM_COL_BITS);
                              if (ii != a.self_img) {
                                  const float4 ph = a.phasedf[ii];
                                  const float pr = ph.x, pi = fs * ph.z;
                                  t = make_float2(pr * t.x - pi * t.y, pr * t.y + pi * t.x);
                              }
                              sr += t.x;
                              si += t.y;
                          });
            two_sum_acc(rh, rl, sr);
            two_sum_acc(ih, il, si);
        } else {
            const float4* vr = a.valdf + r0;
            corr_row<UNR>(lane, len, colr, [=](int e) { return __ldcs(vr + e); }, qs, body);
        }
    } else if (CM == PIM_CORR_FP32) {
        const float2* vr = a.valf + r0;
        corr_row<UNR>(lane, len, colr, [=](int e) { return __ldcs(vr + e); }, qs,
                      [&](uint32_t c, const float2& d, const cplx<T>& x) {
            const float xr = (float)x.x, xi = fs * (float)x.y;
            float2 t = make_float2(d.x * xr - d.y * xi, d.x * xi + d.y * xr);
            const int ii = (int)(c >> PIM_COL_BITS);
            if (ii != a.self_img) {
                const float4 ph = a.phasedf[ii];
                const float pr = ph.x, pi = fs * ph.z;
                t = make_float2(pr * t.x - pi * t.y, pr * t.y + pi * t.x);
            }
            rh += t.x;
            ih += t.y;
        });
    }
    // warp reduction
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
        if (CM == PIM_CORR_FP64) {
            accd.x += __shfl_xor_sync(0xffffffffu, accd.x, o);
            accd.y += __shfl_xor_sync(0xffffffffu, accd.y, o);
        } else if (CM == PIM_CORR_FP32) {
            rh += __shfl_xor_sync(0xffffffffu, rh, o);
            ih += __shfl_xor_sync(0xffffffffu, ih, o);
        }
    }
    if (corr_df(CM)) {
        df_warp_sum(rh, rl);
        df_warp_sum(ih, il);
    }
    if (lane == 0) {
        T re, im;
        if constexpr (sizeof(T) == 4 && CM != PIM_CORR_FP64) {
            // FP32 output: grid part + correction rounded once, without the
            // FP64 pipe (TwoSum of the leading parts, then the tails)
            float s, e;
            ih *= fs;  // undo the conjugation of the adjoint sum
            il *= fs;
            two_sum(acc.x, rh, s, e);
            re = s + (e + rl);
            two_sum(acc.y, ih, s, e);
            im = s + (e + il);
        } else {
            accd.y *= (double)fs;  // undo the conjugation of the adjoint sum
            re = (T)((double)acc.x + accd.x);
            im = (T)((double)acc.y + accd.y);
        }
        if (a.sorted_out) {
            ((cplx<T>*)out)[m] = mk<T>(re, im);
        } else {
            const long long o = (long long)a.perm[m] * a.nrhs + a.r;
            if (a.real_out) ((T*)out)[o] = re;
            else ((cplx<T>*)out)[o] = mk<T>(re, im);
        }
    }
}

// Launch-shape variants of the gather kernel, chosen per plan by the
// autotuner: (unroll depth of the correction loop, minimum resident CTAs).
constexpr int GATHER_VARIANTS = 5;

template <typename T, int PP, int CM>
pim_status launch_gather_cm(int v, unsigned nb, cudaStream_t s, const GatherArgs& ga, const cplx<T>* U,
                            const cplx<T>* qs, void* dst) {
    switch (v) {
        case 0: gather_kernel<T, PP, CM, 2, 6><<<nb, 256, 0, s>>>(ga, U, qs, dst); break;
        case 1: gather_kernel<T, PP, CM, 4, 4><<<nb, 256, 0, s>>>(ga, U, qs, dst); break;
        case 2: gather_kernel<T, PP, CM, 3, 5><<<nb, 256, 0, s>>>(ga, U, qs, dst); break;
        case 3: gather_kernel<T, PP, CM, 2, 8><<<nb, 256, 0, s>>>(ga, U, qs, dst); break;
        default: gather_kernel<T, PP, CM, 1, 8><<<nb, 256, 0, s>>>(ga, U, qs, dst); break;
    }
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <typename T, int PP>
pim_status launch_gather(int cm, int v, unsigned nb, cudaStream_t s, const GatherArgs& ga, const cplx<T>* U,
                         const cplx<T>* qs, void* dst) {
    if (cm < 0) {
        // near and far gathers only (the correction runs in the multi-RHS kernel)
        gather_kernel<T, PP, -1, 1, 8><<<nb, 256, 0, s>>>(ga, U, qs, dst);
        PIM_CK(cudaGetLastError());
        return PIM_OK;
    }
    if constexpr (sizeof(T) == 8) {
        return launch_gather_cm<T, PP, PIM_CORR_FP64>(v, nb, s, ga, U, qs, dst);
    } else {
        if (cm == PIM_CORR_COMPACT) return launch_gather_cm<T, PP, PIM_CORR_COMPACT>(v, nb, s, ga, U, qs, dst);
        if (cm == PIM_CORR_DOUBLE_FLOAT)
            return launch_gather_cm<T, PP, PIM_CORR_DOUBLE_FLOAT>(v, nb, s, ga, U, qs, dst);
        if (cm == PIM_CORR_FP32) return launch_gather_cm<T, PP, PIM_CORR_FP32>(v, nb, s, ga, U, qs, dst);
        return launch_gather_cm<T, PP, PIM_CORR_FP64>(v, nb, s, ga, U, qs, dst);
    }
}

}  // namespace pim_k
