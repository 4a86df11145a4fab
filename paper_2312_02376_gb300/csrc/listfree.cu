// List-free near-pair correction (Sec. 3.3 step 4, Eq. er) for observer boxes
// that hold many points and many correction partners.
//
// For every observer box A the correction region (the boxes within D^ER of
// A, per near image i, as for the stored list) is the same for all points of
// A, and all points of a box share one interpolation stencil.  The correction
// of Eq. er summed over the region,
//
//   c_m = sum_{(n,i) in region(A)} exp(-j k0.(i o L))
//           [ G0(r_m - r_n - i o L) - sum_a sum_c w_m(a) w_n(c) g(a - c - i o (n-1)) ],
//
// splits into an exact part (a direct sum over the region's points) and a
// grid part w_m . V_A with
//
//   V_A(a) = sum_c g(a - c) Q_A(c),
//   Q_A    = sum_{(B,i) in region(A)} exp(-j k0.(i o L)) M_B placed at s_B + i o (n-1),
//
// where M_B(c) = sum_{n in B} w_n(c) q_n are the box moments of step 1 (the
// spread forms them for the boxes with >= PIM_DENSE_MIN points) and g(e) =
// G0(|e o h|), g(0) = 0, is the grid kernel
// of the image-i component (an image shift moves a box by whole periods of
// n - 1 grid steps, so g is the free-space kernel on the unrolled grid).  Only
// the region's boxes with moments take part here: the pairs of A's points with
// the points of the region's other boxes stay in the stored list (few points,
// each spread over a whole stencil, would fill the local grid).  Q_A
// lives on a local grid of E^3 nodes around A in shared memory, so the grid
// part costs one small convolution per box instead of one 729-term sum per
// pair, and nothing is stored between applies.  The adjoint uses conj(G0),
// conj(g) and the same image phases (the region is symmetric), as the stored
// list does.
//
// Local grid frame of box A (per axis): origin A - R - 2c; a box B' = B +
// i (n-1) of the region has |B' - A| <= R and its clamped stencil start s_B
// differs from B - c by at most c, so s_B' - origin lies in [0, 2R + 2c] and
// its stencil in [0, E - 1], E = 2R + 2c + p + 1; A's own stencil starts at
// X0 = s_A - origin in [R, R + 2c]; the offsets a - c reach |e| <= H = R + 2c + p.
#include <algorithm>
#include <cmath>

#include "lagrange.cuh"
#include "pim_internal.cuh"

namespace {
using namespace pim_k;

constexpr double PI = 3.141592653589793238462643383279502884;
constexpr int LF_NT = 256;      // threads of the exact-part kernel
constexpr int LF_CH = 2048;     // region points staged per chunk
constexpr int LF_MAXOBS = 256;  // observers per pass over the region
constexpr int LF_GNT = 512;     // threads of the grid-part kernel
constexpr int LF_MAXNT = 8;     // polynomial terms
constexpr int LF_MAXSEG = 512;  // region segments of a box staged in shared memory

struct LfArgs {
    const int* lfslot;
    const int64_t* segptr;
    const int4* seg;
    const int* lfself;
    const int* lfnear;
    const float4* lfl;
    const int* bstart;
    const int* blist;
    const int* dix;
    const float4* lfp;
    const double* pos;
    const float* nt;
    const double* ntd;
    const int* perm;
    const double2* phase;   // exp(-j k0.(i o L)) per near image
    int nb[3], nL[3], n[3];
    int p, c, R, E, H;
    int nimg, self_img;
    int img[PIM_MAX_IMAGES][3];
    double h[3], D[3];
    float hf[3];
    double k;
    float pc[LF_MAXNT], ps[LF_MAXNT];  // cos and sinc polynomial coefficients (x 1/(4 pi)), in s = r^2
    long long nlf;
    int nrhs, r, real_out, sorted_out;
    int* status;
    unsigned long long* next;   // box counter of the exact-part kernel
    void* ulf;              // exact part: stored here (sorted order) instead of added to the output;
                            // grid part: added to the output with it
    // grid part on the tensor cores: the boxes it handles (tcmask, by list-free
    // index) are skipped by lf_grid_kernel; in its Q-output form the kernel
    // takes the boxes tcl[0, tcrows) and writes their local grids as rows of
    // tcKP-padded FP32 [Re Q | Im Q] to the kernel's out
    const unsigned char* tcmask;
    const int* tcl;
    long long tcrows;
    int tcKP;
};

// an FP64 position padded to 32 bytes
struct __align__(16) dpos4 {
    double x, y, z, w;
};

__device__ __forceinline__ void box_xyz(int b, const int* nb, int* B) {
    B[0] = b % nb[0];
    B[1] = (b / nb[0]) % nb[1];
    B[2] = b / (nb[0] * nb[1]);
}

// stencil start of box B along one axis: clamp(B - c, 0, n - 1 - p)
__device__ __forceinline__ int box_stencil(int B, int c, int n, int p) { return min(max(B - c, 0), n - 1 - p); }

// x rounded to TF32 (10 explicit mantissa bits, to nearest, ties away), held in
// an FP32 register with the low 13 bits zero
__device__ __forceinline__ float tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// dst[m] += v in the layout of the apply's output (caller order with the
// right-hand-side stride, real or complex, or the sorted scratch)
template <typename T>
__device__ __forceinline__ void add_out(const LfArgs& a, void* out, long long m, cplx<T> v) {
    if (a.sorted_out) {
        cplx<T>* u = (cplx<T>*)out + m;
        *u = mk<T>(u->x + v.x, u->y + v.y);
        return;
    }
    const long long o = (long long)a.perm[m] * a.nrhs + a.r;
    if (a.real_out) {
        ((T*)out)[o] += v.x;
    } else {
        cplx<T>* u = (cplx<T>*)out + o;
        *u = mk<T>(u->x + v.x, u->y + v.y);
    }
}

// The region segments of list-free box j in shared memory (a box with more
// segments reads them from global memory), with the first point of each:
// returns the table and sets ns, and sp0 to the point table.
__device__ __forceinline__ const int4* stage_segments(const LfArgs& a, int64_t g0, int64_t g1, int4* sSeg, int* sP0,
                                                      int& ns, const int*& p0) {
    ns = (int)(g1 - g0);
    if (ns > LF_MAXSEG) {
        p0 = nullptr;
        return a.seg + g0;
    }
    for (int i = threadIdx.x; i < ns; i += blockDim.x) {
        const int4 sg = a.seg[g0 + i];
        sSeg[i] = sg;
        if (sP0) sP0[i] = a.bstart[sg.x];
    }
    p0 = sP0;
    return sSeg;
}

// index of the last segment whose offset (point offset w, or slot offset
// z >> 8) is <= f
template <bool SLOTS>
__device__ __forceinline__ int find_segment(const int4* t, int ns, int f) {
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int key = SLOTS ? (t[mid].z >> 8) : t[mid].w;
        if (key <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Reduce-scatter of NV values (8 or 16) over the warp: afterwards lane l
// holds the warp sum of value l >> (5 - log2 NV) (the 32 / NV lanes of a
// group all hold it).
template <int NV>
__device__ __forceinline__ float reduce_scatter(float* v, int lane) {
#pragma unroll
    for (int o = 16, h = NV / 2; h >= 1; o >>= 1, h >>= 1) {
        const bool up = lane & o;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    float r = v[0];
#pragma unroll
    for (int o = 16 / NV; o >= 1; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    return r;
}

// ------------------------------ exact part --------------------------------
// 1/sqrt(x) by the SFU, denormals flushed (PTX rsqrt.approx.ftz.f32, relative
// error about 2^-23): one instruction per pair.
__device__ __forceinline__ float rsqrt_sfu(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// G0 of one pair times its source, added to (ar, ai): s = r^2, q the source
// times its image phase.  NT > 0: cos(k r) / (4 pi) and -k sinc(k r) / (4 pi)
// as polynomials in s (coefficients pc, ps); NT = 0: sincosf.  CHECK: the
// pair may be the point itself (s = 0), which adds nothing.
template <int MODE, int NT, bool CHECK>
__device__ __forceinline__ void g0_val(const LfArgs& a, float s, float& gr, float& gim) {
    float ri = rsqrt_sfu(s);
    if (CHECK) ri = s > 0.f ? ri : 0.f;
    if (NT > 0) {
        float pcv = a.pc[NT - 1], psv = a.ps[NT - 1];
#pragma unroll
        for (int t = NT - 2; t >= 0; --t) {
            pcv = fmaf(pcv, s, a.pc[t]);
            psv = fmaf(psv, s, a.ps[t]);
        }
        gr = ri * pcv;
        gim = CHECK ? (s > 0.f ? psv : 0.f) : psv;
    } else {
        float sn, cs;
        sincosf((float)a.k * (s * ri), &sn, &cs);
        const float s4 = ri * (float)(0.25 / PI);
        gr = cs * s4;
        gim = -sn * s4;
    }
    if (MODE == 1) gim = -gim;
}

template <int MODE, int NT, bool CHECK>
__device__ __forceinline__ void g0_mac(const LfArgs& a, float s, float2 q, float& ar, float& ai) {
    float gr, gim;
    g0_val<MODE, NT, CHECK>(a, s, gr, gim);
    ar = fmaf(gr, q.x, fmaf(-gim, q.y, ar));
    ai = fmaf(gr, q.y, fmaf(gim, q.x, ai));
}

// The staged points [0, cnt) against the observers [0, no): warps split the
// points, lanes take every 32nd of a warp's share, each lane sums LF_OB
// observers at once; the sums are reduced over the warp and added to sAcc.
// PREC: points and observers as double-float coordinates in grid steps
// relative to A's centre (heads sX, sO; tails sX + LF_CH / 2, sOl), their
// differences formed exactly before they are scaled by h; otherwise FP32
// positions in physical units (sX; observers sO scaled by h).
// REV (far chunks of the symmetric form): each source's sum over the
// observers of K q_obs (K = G0, conj for MODE 1) is also formed, per source in
// sRev[s] (each source belongs to one thread for all observer groups).
template <int MODE, int NT, bool CHECK, bool PREC, int LF_OB, int CH, bool REV>
__device__ __forceinline__ void exact_chunk(const LfArgs& a, const float4* sX, const float2* sQ, const float4* sO,
                                            const float4* sOl, float* sAcc, int no, int cnt, int warp, int lane,
                                            const float2* sOq, float2* sRev) {
    constexpr int NV = 2 * LF_OB, SH = NV == 16 ? 1 : 2;   // lane >> SH: the value a lane holds
    const int ngr = (no + LF_OB - 1) / LF_OB;
    const float4* sXl = sX + CH / 2;
    for (int gi = 0; gi < ngr; ++gi) {
        float ox[LF_OB], oy[LF_OB], oz[LF_OB], olx[LF_OB], oly[LF_OB], olz[LF_OB], ar[LF_OB], ai[LF_OB];
#pragma unroll
        for (int k = 0; k < LF_OB; ++k) {
            const int i = gi * LF_OB + k;
            const float4 O = i < no ? sO[i] : make_float4(1e3f, 1e3f, 1e3f, 0.f);
            if (PREC) {
                const float4 Ol = i < no ? sOl[i] : make_float4(0.f, 0.f, 0.f, 0.f);
                ox[k] = O.x;
                oy[k] = O.y;
                oz[k] = O.z;
                olx[k] = Ol.x;
                oly[k] = Ol.y;
                olz[k] = Ol.z;
            } else {
                ox[k] = O.x * a.hf[0];
                oy[k] = O.y * a.hf[1];
                oz[k] = O.z * a.hf[2];
            }
            ar[k] = 0.f;
            ai[k] = 0.f;
        }
        float2 oq[REV ? LF_OB : 1];
        if (REV) {
#pragma unroll
            for (int k = 0; k < LF_OB; ++k) {
                const int i = gi * LF_OB + k;
                oq[k] = i < no ? sOq[i] : make_float2(0.f, 0.f);
            }
        }
        for (int s = warp * 32 + lane; s < cnt; s += LF_NT) {
            const float4 X = sX[s];
            const float2 q = sQ[s];
            float4 Xl;
            if (PREC) Xl = sXl[s];
            float rr = 0.f, rim = 0.f;
#pragma unroll
            for (int k = 0; k < LF_OB; ++k) {
                float dx = ox[k] - X.x, dy = oy[k] - X.y, dz = oz[k] - X.z;
                if (PREC) {
                    // heads of close points differ exactly; add the tails' difference
                    dx = (dx + (olx[k] - Xl.x)) * a.hf[0];
                    dy = (dy + (oly[k] - Xl.y)) * a.hf[1];
                    dz = (dz + (olz[k] - Xl.z)) * a.hf[2];
                }
                if (REV) {
                    float gr, gim;
                    g0_val<MODE, NT, CHECK>(a, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), gr, gim);
                    ar[k] = fmaf(gr, q.x, fmaf(-gim, q.y, ar[k]));
                    ai[k] = fmaf(gr, q.y, fmaf(gim, q.x, ai[k]));
                    rr = fmaf(gr, oq[k].x, fmaf(-gim, oq[k].y, rr));
                    rim = fmaf(gr, oq[k].y, fmaf(gim, oq[k].x, rim));
                } else {
                    g0_mac<MODE, NT, CHECK>(a, fmaf(dx, dx, fmaf(dy, dy, dz * dz)), q, ar[k], ai[k]);
                }
            }
            if (REV) {
                float2 t = sRev[s];
                t.x += rr;
                t.y += rim;
                sRev[s] = t;
            }
        }
        float v[2 * LF_OB];
#pragma unroll
        for (int k = 0; k < LF_OB; ++k) {
            v[2 * k] = ar[k];
            v[2 * k + 1] = ai[k];
        }
        const float sum = reduce_scatter<NV>(v, lane);
        const int vi = lane >> SH;
        const int i = gi * LF_OB + (vi >> 1);
        if (!(lane & ((1 << SH) - 1)) && i < no) atomicAdd(&sAcc[2 * i + (vi & 1)], sum);
    }
}

// One CTA per list-free box.  The region's points are staged in shared
// memory, LF_CH at a time (LF_CH / 2 for the double-float chunks), with their
// source strengths times the image phase, in the order: A's own points
// (image 0; the only chunks that can hold the pair of a point with itself,
// summed with the s > 0 test), the other points of the 27 boxes around A
// (pairs as close as the points come: double-float coordinates in grid steps
// relative to A's centre, the integer box offset and the box-centred
// coordinate added exactly), then the rest of the region (at least one box
// apart: FP32 positions in physical units).  Every pair but a point's own
// has s > 0: set-points rejects points that coincide.
//
// MODE 0: forward, 1: adjoint (conj(G0)), 2: check only (flags pairs of
// distinct points with s = 0).
//
// SYM (one right-hand side, the exact list with flagged segments): beyond the
// 27 boxes a flagged partner box is list-free and keeps no segment of this
// box, so this CTA sums each such pair once for both: K times the source into
// the observer's sum, K times the observer's strength into the source's
// (with the phase of the mirrored image), added to ulf by atomics; ulf is zero
// at launch.  Chunks of 1280 points keep three CTAs per SM.
template <int MODE, int NT, bool SYM = false>
__global__ void __launch_bounds__(LF_NT, 3) lf_exact_f32(LfArgs a, const float2* __restrict__ qs, void* out) {
    constexpr int CH = SYM ? 1280 : LF_CH;
    extern __shared__ __align__(16) unsigned char smem[];
    float4* sX = (float4*)smem;                          // CH
    float2* sQ = (float2*)(sX + CH);                     // CH
    float4* sO = (float4*)(sQ + CH);                     // LF_MAXOBS: heads, grid steps
    float4* sOl = sO + LF_MAXOBS;                        // LF_MAXOBS: tails
    float* sAcc = (float*)(sOl + LF_MAXOBS);             // 2 LF_MAXOBS
    int4* sSeg = (int4*)(sAcc + 2 * LF_MAXOBS);          // LF_MAXSEG
    int* sP0 = (int*)(sSeg + LF_MAXSEG);                 // LF_MAXSEG
    int* sIdx = sP0 + LF_MAXSEG;                         // CH (check mode; SYM: image << 25 | point, or ~0)
    float2* sRev = (float2*)(sIdx + CH);                 // CH (SYM)
    float2* sOq = sRev + CH;                             // LF_MAXOBS (SYM): the observers' strengths
    __shared__ long long sj;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // boxes are taken from a counter (zero at launch): the CTAs stay resident
    // (a set number per SM, leaving room for concurrent kernels) and the
    // boxes' uneven costs balance out
    for (;;) {
        __syncthreads();
        if (tid == 0) sj = (long long)atomicAdd(a.next, 1ULL);
        __syncthreads();
        const long long j = sj;
        if (j >= a.nlf) break;
        const int sA = a.lfslot[j];
        const int m0 = a.bstart[sA], nA = a.bstart[sA + 1] - m0;
        int A[3];
        box_xyz(a.blist[sA], a.nb, A);
        const int64_t g0 = a.segptr[j], g1 = a.segptr[j + 1];
        if (g1 == g0) continue;  // no dense box in the region (uniform over the CTA)
        __syncthreads();
        int ns;
        const int* p0t;
        const int4* tab = stage_segments(a, g0, g1, sSeg, sP0, ns, p0t);
        const int4 last = a.seg[g1 - 1];
        const int total = last.w + (a.bstart[last.y] - a.bstart[last.x]);
        // the region's list: [0, nnear) the 27 boxes around A, with A's own
        // points at [so, so + nA) (so < 0: A has no moments, its pairs with
        // itself are stored); taken as [A's points][the rest of the 27
        // boxes][the others]
        const int so = a.lfself[j], nnear = a.lfnear[j];
        const int nself = so >= 0 ? nA : 0;
        for (int o0 = 0; o0 < nA; o0 += LF_MAXOBS) {
            const int no = min(LF_MAXOBS, nA - o0);
            __syncthreads();
            for (int i = tid; i < no; i += LF_NT) {
                const float4 L = a.lfp[m0 + o0 + i];
                sO[i] = make_float4(L.x, L.y, L.z, 0.f);
                sOl[i] = a.lfl[m0 + o0 + i];
                sAcc[2 * i] = 0.f;
                sAcc[2 * i + 1] = 0.f;
                if (SYM) sOq[i] = qs[m0 + o0 + i];
            }
            int v0 = 0;
            while (v0 < total) {
                const bool own = v0 < nself, prec = v0 < nnear;
                const int vend = own ? nself : (prec ? nnear : total);
                const int cnt = min(prec ? CH / 2 : CH, vend - v0);
                __syncthreads();
                // stage: every thread finds the segment of each of its points
                // (binary search) and loads it, the loads of all in flight
#pragma unroll 4
                for (int t = tid; t < cnt; t += LF_NT) {
                    const int v = v0 + t;
                    int f = v;
                    if (own) f = so + v;
                    else if (prec && so >= 0) f = v - nself < so ? v - nself : v;
                    const int gs = find_segment<false>(tab, ns, f);
                    const int4 sg = tab[gs];
                    const int nn = (p0t ? p0t[gs] : a.bstart[sg.x]) + (f - sg.w);
                    const int ii = sg.z & 127;
                    const float4 L = a.lfp[nn];
                    int Bn[3];
                    unpack3(__float_as_uint(L.w), Bn[0], Bn[1], Bn[2]);
                    const float bx = (float)(Bn[0] + a.img[ii][0] * a.nL[0] - A[0]);
                    const float by = (float)(Bn[1] + a.img[ii][1] * a.nL[1] - A[1]);
                    const float bz = (float)(Bn[2] + a.img[ii][2] * a.nL[2] - A[2]);
                    if (prec) {
                        // integer offset + head exactly: s + e (|offset| >= |head| or offset 0)
                        const float4 Ll = a.lfl[nn];
                        const float sx = bx + L.x, sy = by + L.y, sz = bz + L.z;
                        sX[t] = make_float4(sx, sy, sz, 0.f);
                        sX[CH / 2 + t] = make_float4((L.x - (sx - bx)) + Ll.x, (L.y - (sy - by)) + Ll.y,
                                                     (L.z - (sz - bz)) + Ll.z, 0.f);
                    } else {
                        sX[t] = make_float4((bx + L.x) * a.hf[0], (by + L.y) * a.hf[1], (bz + L.z) * a.hf[2], 0.f);
                        if (SYM) {
                            ((unsigned*)sIdx)[t] = (sg.z & 128) ? ((unsigned)ii << 25) | (unsigned)nn : 0xFFFFFFFFu;
                            sRev[t] = make_float2(0.f, 0.f);
                        }
                    }
                    if (MODE == 2) {
                        sIdx[t] = ii == a.self_img ? nn : -1;
                    } else {
                        const double2 phd = a.phase[ii];
                        const float2 ph = make_float2((float)phd.x, (float)phd.y);
                        const float2 q = qs[nn];
                        sQ[t] = make_float2(q.x * ph.x - q.y * ph.y, q.x * ph.y + q.y * ph.x);
                    }
                }
                __syncthreads();
                if (MODE == 2) {
                    for (int w = tid; w < no * cnt; w += LF_NT) {
                        const int i = w / cnt, s = w - i * cnt;
                        const float4 O = sO[i], X = sX[s];
                        float dx = O.x - X.x, dy = O.y - X.y, dz = O.z - X.z;
                        if (prec) {
                            const float4 Ol = sOl[i], Xl = sX[CH / 2 + s];
                            dx += Ol.x - Xl.x;
                            dy += Ol.y - Xl.y;
                            dz += Ol.z - Xl.z;
                        } else {
                            dx = O.x * a.hf[0] - X.x;
                            dy = O.y * a.hf[1] - X.y;
                            dz = O.z * a.hf[2] - X.z;
                        }
                        if (dx * dx + dy * dy + dz * dz == 0.f && sIdx[s] != m0 + o0 + i)
                            atomicOr(a.status, PIM_DEV_COINCIDENT);
                    }
                } else if (own) {
                    exact_chunk<MODE, NT, true, true, 4, CH, false>(a, sX, sQ, sO, sOl, sAcc, no, cnt, warp, lane, sOq,
                                                                    sRev);
                } else if (prec) {
                    exact_chunk<MODE, NT, false, true, 4, CH, false>(a, sX, sQ, sO, sOl, sAcc, no, cnt, warp, lane, sOq,
                                                                     sRev);
                } else {
                    exact_chunk<MODE, NT, false, false, 8, CH, SYM>(a, sX, sQ, sO, sOl, sAcc, no, cnt, warp, lane, sOq,
                                                                    sRev);
                    if (SYM) {
                        // the sources' sums, with the phase of the mirrored image,
                        // into their own outputs (other CTAs add to them as well)
                        __syncthreads();
                        for (int t = tid; t < cnt; t += LF_NT) {
                            const unsigned code = ((const unsigned*)sIdx)[t];
                            if (code == 0xFFFFFFFFu) continue;
                            const int nn = (int)(code & 0x1FFFFFFu), ii = (int)(code >> 25);
                            const double2 phd = a.phase[a.nimg - 1 - ii];
                            const float2 S = sRev[t];
                            const float px = (float)phd.x, py = (float)phd.y;
                            atomicAdd((float*)a.ulf + 2 * (long long)nn, px * S.x - py * S.y);
                            atomicAdd((float*)a.ulf + 2 * (long long)nn + 1, px * S.y + py * S.x);
                        }
                    }
                }
                v0 += cnt;
            }
            __syncthreads();
            if (MODE != 2)
                for (int i = tid; i < no; i += LF_NT) {
                    const float2 v = make_float2(sAcc[2 * i], sAcc[2 * i + 1]);
                    if (SYM) {
                        atomicAdd((float*)a.ulf + 2 * (long long)(m0 + o0 + i), v.x);
                        atomicAdd((float*)a.ulf + 2 * (long long)(m0 + o0 + i) + 1, v.y);
                    } else if (a.ulf) {
                        ((float2*)a.ulf)[m0 + o0 + i] = v;
                    } else {
                        add_out<float>(a, out, m0 + o0 + i, v);
                    }
                }
        }
    }
}

// The same in FP64 from the FP64 positions (one source per lane, no staging of
// observers in registers: FP64 plans are for accuracy, not speed).
template <int MODE>
__global__ void __launch_bounds__(LF_NT) lf_exact_f64(LfArgs a, const double2* __restrict__ qs, void* out) {
    extern __shared__ __align__(16) unsigned char smem[];
    dpos4* sX = (dpos4*)smem;                        // LF_CH
    double2* sQ = (double2*)(sX + LF_CH);                // LF_CH
    int* sIdx = (int*)(sQ + LF_CH);                      // LF_CH
    int4* sSeg = (int4*)(sIdx + LF_CH);                  // LF_MAXSEG
    int* sP0 = (int*)(sSeg + LF_MAXSEG);                 // LF_MAXSEG
    const int tid = threadIdx.x;
    for (long long j = blockIdx.x; j < a.nlf; j += gridDim.x) {
        const int sA = a.lfslot[j];
        const int m0 = a.bstart[sA], nA = a.bstart[sA + 1] - m0;
        const int64_t g0 = a.segptr[j], g1 = a.segptr[j + 1];
        if (g1 == g0) continue;  // no dense box in the region (uniform over the CTA)
        __syncthreads();
        int ns;
        const int* p0t;
        const int4* tab = stage_segments(a, g0, g1, sSeg, sP0, ns, p0t);
        const int4 last = a.seg[g1 - 1];
        const int total = last.w + (a.bstart[last.y] - a.bstart[last.x]);
        // thread t sums observer t % nA over the staged points t / nA, + LF_NT / nA ...
        const int per = max(1, LF_NT / max(nA, 1));
        for (int o0 = 0; o0 < nA; o0 += LF_NT) {
            const int no = min(nA - o0, LF_NT);
            const int stride = no < LF_NT ? per : 1;
            const int i = tid % no, part = tid / no;
            const bool act = part < stride;
            const long long m = m0 + o0 + i;
            const double px = a.pos[3 * m], py = a.pos[3 * m + 1], pz = a.pos[3 * m + 2];
            double2 acc = make_double2(0.0, 0.0);
            for (int f0 = 0; f0 < total; f0 += LF_CH) {
                const int cnt = min(LF_CH, total - f0);
                __syncthreads();
                for (int t = tid; t < cnt; t += LF_NT) {
                    const int f = f0 + t;
                    const int gs = find_segment<false>(tab, ns, f);
                    const int4 sg = tab[gs];
                    const int nn = (p0t ? p0t[gs] : a.bstart[sg.x]) + (f - sg.w);
                    const int ii = sg.z & 255;
                    sX[t] = dpos4{a.pos[3 * nn] + a.img[ii][0] * a.D[0], a.pos[3 * nn + 1] + a.img[ii][1] * a.D[1],
                                 a.pos[3 * nn + 2] + a.img[ii][2] * a.D[2], 0.0};
                    sIdx[t] = ii == a.self_img ? nn : -1;
                    if (MODE != 2) sQ[t] = cmul(qs[nn], a.phase[ii]);
                }
                __syncthreads();
                if (!act) continue;
                for (int s = part; s < cnt; s += stride) {
                    const dpos4 X = sX[s];
                    const double dx = px - X.x, dy = py - X.y, dz = pz - X.z;
                    const double r2 = dx * dx + dy * dy + dz * dz;
                    if (r2 == 0.0) {
                        if (MODE == 2 && sIdx[s] != m) atomicOr(a.status, PIM_DEV_COINCIDENT);
                        continue;
                    }
                    if (MODE == 2) continue;
                    const double R = sqrt(r2);
                    double sn, cs;
                    sincos(a.k * R, &sn, &cs);
                    const double s4 = 1.0 / (4.0 * PI * R);
                    const double2 G = make_double2(cs * s4, (MODE == 1 ? sn : -sn) * s4);
                    acc = cadd(acc, cmul(G, sQ[s]));
                }
            }
            __syncthreads();
            // sum the parts of each observer in shared memory (reusing sQ)
            if (MODE != 2) {
                if (act) sQ[part * no + i] = acc;
                __syncthreads();
                if (tid < no) {
                    double2 t = make_double2(0.0, 0.0);
                    for (int k = 0; k < stride; ++k) t = cadd(t, sQ[k * no + tid]);
                    if (a.ulf) ((double2*)a.ulf)[m0 + o0 + tid] = t;
                    else add_out<double>(a, out, m0 + o0 + tid, t);
                }
            }
        }
    }
}

// ------------------------------ grid part ---------------------------------
// One CTA per list-free box:
//  1. a table of the region's dense boxes in shared memory (moment index,
//     position of the stencil in the local grid, image), LF_MAXSLOT boxes at
//     a time;
//  2. their moments, times the image phase, are added into the local grid
//     Q_A (shared-memory atomics), work item = (region box, stencil row
//     (jy, jz)); each x-row of Q_A records the x-range it received;
//  3. V_A = g * Q_A at A's own (P+1)^3 stencil nodes: warps take the
//     non-empty x-rows of Q_A, lane (ay, az) one output x-row; per block of 8
//     input nodes inside the row's x-range the lane holds the g values of
//     8 + P x-offsets in registers and does (P+1) x 8 complex multiply-adds;
//     the warps' sums meet in shared memory (atomics);
//  4. every point of A subtracts w_m . V_A from its output.
// The kernel table g(|e|) ((H+1)^3 entries) sits in shared memory for FP32
// plans: the lanes of a warp read 25 different rows of it, a few bank
// conflicts there instead of as many cache lines through L1.
constexpr int LF_MAXSLOT = 1024;

// OUTQ: the Q-output form (steps 1 and 2 only; tensor-core path).
template <typename T, int P, int EX, bool ADJ, bool OUTQ = false>
__global__ void __launch_bounds__(LF_GNT) lf_grid_kernel(LfArgs a, const cplx<T>* __restrict__ mom,
                                                       const cplx<T>* __restrict__ gtab, void* out) {
    constexpr int NP = P + 1, RW = NP * NP, NW = LF_GNT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int E = a.E, H1 = a.H + 1;
    constexpr int XS = EX + 1;                               // row stride (odd: rows in different banks)
    const int ncell = E * E * XS;
    cplx<T>* Q = (cplx<T>*)smem;                             // E x E rows of XS
    T* Vr = (T*)(Q + ncell);                                 // NP^3
    T* Vi = Vr + NP * NP * NP;                               // NP^3
    int2* slot = (int2*)(((uintptr_t)(Vi + NP * NP * NP) + 15) & ~(uintptr_t)15);  // LF_MAXSLOT
    int* xlo = (int*)(slot + LF_MAXSLOT);                    // E^2
    int* xhi = xlo + E * E;                                  // E^2
    int* rows = xhi + E * E;                                 // E^2
    int* nrows = rows + E * E;                               // 1
    cplx<T>* gs = (cplx<T>*)(((uintptr_t)(nrows + 1) + 15) & ~(uintptr_t)15);  // H1^3 (FP32)
    const cplx<T>* gt = sizeof(T) == 4 ? gs : gtab;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (sizeof(T) == 4 && !OUTQ)
        for (int i = tid; i < H1 * H1 * H1; i += LF_GNT) {
            cplx<T> g = gtab[i];
            if (ADJ) g.y = -g.y;
            gs[i] = g;
        }
    const long long nbox = OUTQ ? a.tcrows : a.nlf;
    for (long long jj = blockIdx.x; jj < nbox; jj += gridDim.x) {
        const long long j = OUTQ ? (long long)a.tcl[jj] : jj;
        if (!OUTQ && a.tcmask && a.tcmask[j]) continue;  // on the tensor cores
        const int sA = a.lfslot[j];
        const int m0 = a.bstart[sA], nA = a.bstart[sA + 1] - m0;
        int A[3], org[3], X0[3];
        box_xyz(a.blist[sA], a.nb, A);
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            org[d] = A[d] - a.R - 2 * a.c;
            X0[d] = box_stencil(A[d], a.c, a.n[d], a.p) - org[d];
        }
        const int64_t g0 = a.segptr[j], g1 = a.segptr[j + 1];
        if (g1 == g0) continue;  // no dense box in the region (uniform over the CTA)
        __syncthreads();
        for (int i = tid; i < ncell; i += LF_GNT) Q[i] = mk<T>(T(0), T(0));
        for (int i = tid; i < E * E; i += LF_GNT) {
            xlo[i] = EX;
            xhi[i] = -1;
        }
        for (int i = tid; i < NP * NP * NP; i += LF_GNT) {
            Vr[i] = T(0);
            Vi[i] = T(0);
        }
        const int4 last = a.seg[g1 - 1];
        const int nslots = (last.z >> 8) + (last.y - last.x);
        for (int w0 = 0; w0 < nslots; w0 += LF_MAXSLOT) {
            const int nw = min(LF_MAXSLOT, nslots - w0);
            __syncthreads();
            // 1. the window's dense boxes: warps over segments, lanes over slots
            for (int64_t g = g0 + warp; g < g1; g += NW) {
                const int4 sg = a.seg[g];
                const int soff = sg.z >> 8, ii = sg.z & 255;
                const int lo = max(sg.x, sg.x + (w0 - soff)), hi = min(sg.y, sg.x + (w0 + nw - soff));
                for (int sl = lo + lane; sl < hi; sl += 32) {
                    int B[3], loc[3];
                    box_xyz(a.blist[sl], a.nb, B);
                    bool ok = true;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        loc[d] = box_stencil(B[d], a.c, a.n[d], a.p) + a.img[ii][d] * a.nL[d] - org[d];
                        ok = ok && loc[d] >= 0 && loc[d] + P < E;
                    }
                    const int di = a.dix[sl];
                    if (!ok || di < 0) atomicOr(a.status, PIM_DEV_BOUNDS);
                    slot[soff + (sl - sg.x) - w0] =
                        make_int2(ok ? di : -1, loc[0] | (loc[1] << 5) | (loc[2] << 10) | (ii << 15));
                }
            }
            __syncthreads();
            // 2. their moments into the local grid (consecutive lanes take
            // different boxes, so that their atomics fall in different banks)
#pragma unroll 4
            for (int w = tid; w < nw * RW; w += LF_GNT) {
                const int rr = w / nw, f = w - rr * nw;
                const int gy = rr % NP, gz = rr / NP;
                const int2 e = slot[f];
                if (e.x < 0) continue;
                const int lx = e.y & 31, ly = (e.y >> 5) & 31, lz = (e.y >> 10) & 31, ii = e.y >> 15;
                const cplx<T>* mr = mom + (((long long)e.x * NP + gz) * NP + gy) * NP;
                cplx<T> v[NP];
#pragma unroll
                for (int jx = 0; jx < NP; ++jx) v[jx] = mr[jx];
                const double2 phd = a.phase[ii];
                const cplx<T> ph = mk<T>((T)phd.x, (T)phd.y);
                const int row = (lz + gz) * E + (ly + gy);
                cplx<T>* qrow = Q + row * XS + lx;
#pragma unroll
                for (int jx = 0; jx < NP; ++jx) {
                    const cplx<T> x = cmul(v[jx], ph);
                    atomicAdd(&qrow[jx].x, x.x);
                    atomicAdd(&qrow[jx].y, x.y);
                }
                atomicMin(&xlo[row], lx);
                atomicMax(&xhi[row], lx + P);
            }
        }
        __syncthreads();
        if (OUTQ) {
            // the local grid as one FP32 row [Re Q | Im Q] (local node
            // (z E + y) E + x, zero beyond E^3)
            float* bq = (float*)out + (size_t)jj * 2 * a.tcKP;
            const int E3 = E * E * E;
            for (int i = tid; i < a.tcKP; i += LF_GNT) {
                float re = 0.f, im = 0.f;
                if (i < E3) {
                    const cplx<T> v = Q[(i / E) * XS + i % E];
                    re = (float)v.x;
                    im = (float)v.y;
                }
                bq[i] = re;
                bq[a.tcKP + i] = im;
            }
            continue;
        }
        // non-empty rows, in order
        if (warp == 0) {
            int base = 0;
            for (int r0 = 0; r0 < E * E; r0 += 32) {
                const bool f = r0 + lane < E * E && xhi[r0 + lane] >= 0;
                const unsigned b = __ballot_sync(0xffffffffu, f);
                if (f) rows[base + __popc(b & ((1u << lane) - 1u))] = r0 + lane;
                base += __popc(b);
            }
            if (lane == 0) *nrows = base;
        }
        __syncthreads();
        // 3. V_A = g * Q_A at A's stencil nodes
        if (lane < RW) {
            cplx<T> acc[NP];
#pragma unroll
            for (int jx = 0; jx < NP; ++jx) acc[jx] = mk<T>(T(0), T(0));
            const int oy = X0[1] + lane % NP, oz = X0[2] + lane / NP;
            const int nr = *nrows;
            for (int ri = warp; ri < nr; ri += NW) {
                const int row = rows[ri];
                const int cy = row % E, cz = row / E;
                const cplx<T>* grow = gt + ((long long)abs(oz - cz) * H1 + abs(oy - cy)) * H1;
                const cplx<T>* qrow = Q + row * XS;
                const int cend = xhi[row];
                // input nodes cb..cb+7: output jx and input cb + i are
                // e = X0 + jx - cb - i apart, held as gb[jx - i + 7]
#pragma unroll 1
                for (int cb = xlo[row] & ~7; cb <= cend; cb += 8) {
                    cplx<T> gb[8 + P];
#pragma unroll
                    for (int k = 0; k < 8 + P; ++k) {
                        gb[k] = grow[min(abs(X0[0] - cb - 7 + k), a.H)];
                        if (ADJ && sizeof(T) == 8) gb[k].y = -gb[k].y;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const cplx<T> x = qrow[cb + i];
#pragma unroll
                        for (int jx = 0; jx < NP; ++jx) {
                            const cplx<T> g = gb[jx - i + 7];
                            acc[jx].x = fma(g.x, x.x, fma(-g.y, x.y, acc[jx].x));
                            acc[jx].y = fma(g.x, x.y, fma(g.y, x.x, acc[jx].y));
                        }
                    }
                }
            }
            if (nr > warp) {
#pragma unroll
                for (int jx = 0; jx < NP; ++jx) {
                    atomicAdd(Vr + lane * NP + jx, acc[jx].x);
                    atomicAdd(Vi + lane * NP + jx, acc[jx].y);
                }
            }
        }
        __syncthreads();
        // 4. the grid part of every point of A
        for (int i = tid; i < nA; i += LF_GNT) {
            // V is re-read per point: hoisting its NP^3 values out of this
            // loop would not fit in registers
            asm volatile("" ::: "memory");
            const long long m = m0 + i;
            T t[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) t[d] = sizeof(T) == 8 ? (T)a.ntd[3 * m + d] : (T)a.nt[3 * m + d];
            T wx[NP], wy[NP], wz[NP];
            lagrange_w<T, P>(t[0], wx);
            lagrange_w<T, P>(t[1], wy);
            lagrange_w<T, P>(t[2], wz);
            cplx<T> gsum = mk<T>(T(0), T(0));
#pragma unroll
            for (int jz = 0; jz < NP; ++jz)
#pragma unroll
                for (int jy = 0; jy < NP; ++jy) {
                    cplx<T> r = mk<T>(T(0), T(0));
#pragma unroll
                    for (int jx = 0; jx < NP; ++jx) {
                        const int v = (jz * NP + jy) * NP + jx;
                        r.x += wx[jx] * Vr[v];
                        r.y += wx[jx] * Vi[v];
                    }
                    const T w = wy[jy] * wz[jz];
                    gsum.x += w * r.x;
                    gsum.y += w * r.y;
                }
            cplx<T> v = mk<T>(-gsum.x, -gsum.y);
            if (a.ulf) v = cadd(v, ((const cplx<T>*)a.ulf)[m]);
            add_out<T>(a, out, m, v);
        }
    }
}

// ------------------- grid part on the tensor cores -------------------------
// For a box A whose stencil is not clamped at a face of the grid, step 3 of the
// grid part, V_A(s) = sum_nu g(X0 + s - nu) Q_A(nu), uses the same operator for
// every box (X0 = R + c on every axis): one product V = G Q over all such boxes,
// G the 125 x E^3 complex Toeplitz block written in real form as the 256 x 2KP
// matrix [[Re g, -Im g], [Im g, Re g]] (rows: Re V at s, Im V at 128 + s;
// columns [Re Q | Im Q], each padded to KP), Q one row per box.  It runs as a
// tcgen05 kind::tf32 GEMM (accumulators in tensor memory) with each FP32
// operand split into TF32 hi and lo parts, hi.hi + hi.lo + lo.hi (FP32
// accuracy: the dropped lo.lo term is 2^-22 relative).  A CTA takes 128
// boxes (two M = 128 accumulators of 128 columns), K in chunks of 32 staged in
// shared memory in the 128-byte-swizzled K-major layout, two stages: the
// threads load chunk k + 1 while the MMAs of chunk k run.
constexpr int TC_M = 256, TC_N = 128, TC_K = 32, TC_NT = 128;
constexpr int TC_ABYTES = TC_M * TC_K * 4, TC_BBYTES = TC_N * TC_K * 4;
constexpr int TC_STAGE = 2 * TC_ABYTES + 2 * TC_BBYTES;
constexpr size_t TC_SMEM = 2 * (size_t)TC_STAGE + 1024 + 64;
constexpr long long TC_BATCH = 131072;  // boxes per batch (their FP32 Q rows: 131072 x 2KP x 4 bytes)

__device__ __forceinline__ uint32_t tc_saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading byte offset 16
// (unused by the swizzled K-major layout), stride byte offset 1024 (8 rows of
// 128 bytes), descriptor version 1, 128-byte swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                 :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// bounded wait for the completion of phase `parity` of an mbarrier
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
        if (ok) return true;
    }
    return false;
}

// 16-byte asynchronous global -> shared copy; src_bytes 0 fills zeros
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" :: "r"(dst), "l"(src), "r"(src_bytes) : "memory");
}

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled K-major tile
__device__ __forceinline__ uint32_t tc_sw(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

// C[n][m] = sum_k A[m][k] B[n][k] (A: 256 x K, B: N x K, both K-major, each as
// TF32 hi and lo arrays; K a multiple of 32).  On a wait that runs out the
// CTA sets PIM_DEV_TIMEOUT and writes nothing.
__global__ void __launch_bounds__(TC_NT, 1) lf_tc_gemm_kernel(const float* __restrict__ Ah, const float* __restrict__ Al,
                                                             const float* __restrict__ Bq, int K, long long N,
                                                             float* __restrict__ C, int* status) {
    extern __shared__ unsigned char tc_raw[];
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = (uint64_t*)(sm + 2 * TC_STAGE);
    uint32_t* holder = (uint32_t*)(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long n0 = (long long)blockIdx.x * TC_N;
    if (tid == 0) {
        for (int st = 0; st < 2; ++st) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_saddr(bars + st)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" :: "r"(tc_saddr(holder)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *holder;
    // D F32, A and B TF32, both K-major, N = 128, M = 128
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const int nk = K / TC_K;
    uint32_t used[2] = {0, 0};
    bool ok = true;
    // chunk kc into stage st: the operator's hi and lo parts by 16-byte
    // asynchronous copies into the swizzled layout (one commit group per
    // chunk); the FP32 Q rows through registers (all of a thread's loads in
    // flight at once), split into TF32 hi and lo parts on the way (rows past N
    // zero)
    constexpr int BPT = TC_N * 8 / TC_NT;  // 16-byte pieces of B per thread and chunk
    auto load_chunk = [&](int kc, int st) {
        unsigned char* sA = sm + st * TC_STAGE;
        unsigned char* sAl = sA + TC_ABYTES;
        unsigned char* sB = sA + 2 * TC_ABYTES;
        unsigned char* sBl = sB + TC_BBYTES;
        const size_t k0 = (size_t)kc * TC_K;
        for (int e = tid; e < TC_M * 8; e += TC_NT) {
            const int r = e >> 3, c = e & 7;
            cp_async16(tc_saddr(sA + tc_sw(r, c)), Ah + (size_t)r * K + k0 + 4 * c, 16);
            cp_async16(tc_saddr(sAl + tc_sw(r, c)), Al + (size_t)r * K + k0 + 4 * c, 16);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
        float4 v[BPT];
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int e = tid + i * TC_NT, r = e >> 3, c = e & 7;
            const long long n = n0 + r;
            v[i] = n < N ? __ldcs((const float4*)(Bq + (size_t)n * K + k0) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            const int e = tid + i * TC_NT, r = e >> 3, c = e & 7;
            const float4 h = make_float4(tf32_rna(v[i].x), tf32_rna(v[i].y), tf32_rna(v[i].z), tf32_rna(v[i].w));
            const float4 l = make_float4(tf32_rna(v[i].x - h.x), tf32_rna(v[i].y - h.y), tf32_rna(v[i].z - h.z),
                                         tf32_rna(v[i].w - h.w));
            *(float4*)(sB + tc_sw(r, c)) = h;
            *(float4*)(sBl + tc_sw(r, c)) = l;
        }
    };
    if (nk > 0) load_chunk(0, 0);
    for (int kc = 0; kc < nk && ok; ++kc) {
        const int st = kc & 1;
        // the copies of chunk kc (the only group in flight) are in shared
        // memory; make them visible to the tensor cores
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            unsigned char* sA = sm + st * TC_STAGE;
            unsigned char* sAl = sA + TC_ABYTES;
            unsigned char* sB = sA + 2 * TC_ABYTES;
            unsigned char* sBl = sB + TC_BBYTES;
            for (int h = 0; h < 2; ++h) {
                const uint32_t d = tmem + h * TC_N;
                for (int kk = 0; kk < TC_K / 8; ++kk) {
                    const uint32_t ao = h * 128 * 128 + kk * 32, bo = kk * 32;
                    tc_mma(d, tc_desc(tc_saddr(sA) + ao), tc_desc(tc_saddr(sB) + bo), idesc, kc > 0 || kk > 0);
                    tc_mma(d, tc_desc(tc_saddr(sA) + ao), tc_desc(tc_saddr(sBl) + bo), idesc, 1);
                    tc_mma(d, tc_desc(tc_saddr(sAl) + ao), tc_desc(tc_saddr(sB) + bo), idesc, 1);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(tc_saddr(bars + st)));
        }
        if (kc + 1 < nk) {
            // the other stage is free once the MMAs of chunk kc - 1 are done;
            // its copies for chunk kc + 1 then overlap the MMAs of chunk kc
            const int sn = st ^ 1;
            if (kc >= 1) {
                if (!tc_wait(tc_saddr(bars + sn), used[sn] & 1)) ok = false;
                used[sn]++;
            }
            if (ok) load_chunk(kc + 1, sn);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // the last commit of each stage (every earlier one has been waited for)
    for (int st = 0; st < 2 && ok; ++st) {
        const int issued = nk > st ? (nk - st + 1) / 2 : 0;
        if ((int)used[st] < issued) {
            if (!tc_wait(tc_saddr(bars + st), used[st] & 1)) ok = false;
            used[st]++;
        }
    }
    if (!ok) {
        // a wait ran out: wait (bounded) for what was issued, so that the
        // tensor memory is no longer written, then free it
        for (int st = 0; st < 2; ++st) {
            const int issued = nk > st ? (nk - st + 1) / 2 : 0;
            while ((int)used[st] < issued && tc_wait(tc_saddr(bars + st), used[st] & 1)) used[st]++;
        }
        if (tid == 0) atomicOr(status, PIM_DEV_TIMEOUT);
    }
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        for (int h = 0; h < 2; ++h)
            for (int j = 0; j < TC_N / 16; ++j) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + h * TC_N + j * 16;
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                               "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                               "=r"(v[15])
                             : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                const int m = h * 128 + warp * 32 + lane;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const long long n = n0 + j * 16 + i;
                    if (n < N) C[(size_t)n * TC_M + m] = __uint_as_float(v[i]);
                }
            }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem));
}

// The operator of the tensor-core grid part, forward and adjoint (conj g),
// each as TF32 hi and lo parts, from G0 evaluated in FP64.
__global__ void lf_tc_table_kernel(float* Afh, float* Afl, float* Aah, float* Aal, int E, int KP, int X0, int NP, double h0,
                                   double h1, double h2, double k) {
    const long long K2 = 2LL * KP, tot = (long long)TC_M * K2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(e / K2), col = (int)(e % K2);
        const int hh = m / 128, sn = m % 128, part = col / KP, nu = col % KP;
        double gr = 0.0, gi = 0.0;
        if (sn < NP * NP * NP && nu < E * E * E) {
            const int ex = X0 + sn % NP - nu % E, ey = X0 + (sn / NP) % NP - (nu / E) % E,
                      ez = X0 + sn / (NP * NP) - nu / (E * E);
            const double r = sqrt((ex * h0) * (ex * h0) + (ey * h1) * (ey * h1) + (ez * h2) * (ez * h2));
            if (r > 0.0) {
                double sv, cv;
                sincos(k * r, &sv, &cv);
                gr = cv / (4.0 * PI * r);
                gi = -sv / (4.0 * PI * r);
            }
        }
        const double vf = hh == 0 ? (part == 0 ? gr : -gi) : (part == 0 ? gi : gr);
        const double va = hh == 0 ? (part == 0 ? gr : gi) : (part == 0 ? -gi : gr);  // conj g
        const float fh = tf32_rna((float)vf), ah = tf32_rna((float)va);
        Afh[e] = fh;
        Afl[e] = tf32_rna((float)(vf - (double)fh));
        Aah[e] = ah;
        Aal[e] = tf32_rna((float)(va - (double)ah));
    }
}

// Step 4 for the tensor-core boxes: every point of box tcl[row] subtracts
// w_m . V (V = C[row][0..NP^3) + j C[row][128..]), one warp per box.
template <int P>
__global__ void lf_tc_interp_kernel(LfArgs a, const int* __restrict__ tcl, long long rows, const float* __restrict__ C,
                                    void* out) {
    constexpr int NP = P + 1;
    __shared__ float sV[8][TC_M];  // the box's products, one slot per warp (blocks of 256 threads)
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float* V = sV[wib];
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long row = w0; row < rows; row += nw) {
        const int sA = a.lfslot[tcl[row]];
        const int m0 = a.bstart[sA], m1 = a.bstart[sA + 1];
        __syncwarp();
        for (int i = lane; i < TC_M; i += 32) V[i] = __ldg(C + (size_t)row * TC_M + i);
        __syncwarp();
        for (int m = m0 + lane; m < m1; m += 32) {
            float wx[NP], wy[NP], wz[NP];
            lagrange_w<float, P>(a.nt[3 * (long long)m], wx);
            lagrange_w<float, P>(a.nt[3 * (long long)m + 1], wy);
            lagrange_w<float, P>(a.nt[3 * (long long)m + 2], wz);
            float gr = 0.f, gi = 0.f;
#pragma unroll 1
            for (int jz = 0; jz < NP; ++jz)
#pragma unroll
                for (int jy = 0; jy < NP; ++jy) {
                    float rr = 0.f, ri = 0.f;
#pragma unroll
                    for (int jx = 0; jx < NP; ++jx) {
                        const int v = (jz * NP + jy) * NP + jx;
                        rr += wx[jx] * V[v];
                        ri += wx[jx] * V[128 + v];
                    }
                    const float w = wy[jy] * wz[jz];
                    gr += w * rr;
                    gi += w * ri;
                }
            add_out<float>(a, out, m, make_float2(-gr, -gi));
        }
    }
}

// interior list-free boxes with a region: flag and list them
__global__ void lf_tc_list_kernel(const int* lfslot, const int* blist, const int64_t* segptr, long long nlf, int nb0, int nb1,
                                  int n0, int n1, int n2, int c, int p, int X0, int R, unsigned char* mask, int* list,
                                  int* count) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nlf; j += (long long)gridDim.x * blockDim.x) {
        const int b = blist[lfslot[j]];
        const int A[3] = {b % nb0, (b / nb0) % nb1, b / (nb0 * nb1)};
        const int n[3] = {n0, n1, n2};
        bool in = segptr[j + 1] > segptr[j];
        for (int d = 0; d < 3; ++d) in = in && (min(max(A[d] - c, 0), n[d] - 1 - p) - (A[d] - R - 2 * c) == X0);
        mask[j] = in ? 1 : 0;
        if (in) list[atomicAdd(count, 1)] = (int)j;
    }
}

// out += ulf for the points of the list-free boxes (one warp per box), after
// the grid part has been subtracted from ulf on the list-free stream; boxes
// whose region holds no dense box are skipped, as both list-free kernels skip
// them (their ulf entries are not written)
template <typename T>
__global__ void lf_add_kernel(LfArgs a, const cplx<T>* __restrict__ ulf, void* out) {
    const int lane = threadIdx.x & 31;
    const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long j = w0; j < a.nlf; j += nw) {
        if (a.segptr[j + 1] == a.segptr[j]) continue;  // no dense box in its region: nothing was summed
        const int sA = a.lfslot[j];
        const int m0 = a.bstart[sA], m1 = a.bstart[sA + 1];
        for (int m = m0 + lane; m < m1; m += 32) add_out<T>(a, out, m, ulf[m]);
    }
}

// g(|e|) on the offsets 0..H per axis: G0(|e o h|), g(0) = 0 (the grid
// kernel of the near table at zero offset)
template <typename T>
__global__ void lf_table_kernel(cplx<T>* g, int H, double h0, double h1, double h2, double k) {
    const int H1 = H + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < H1 * H1 * H1; e += gridDim.x * blockDim.x) {
        const int x = e % H1, y = (e / H1) % H1, z = e / (H1 * H1);
        const double r = sqrt((x * h0) * (x * h0) + (y * h1) * (y * h1) + (z * h2) * (z * h2));
        double sn = 0.0, cs = 0.0;
        if (r > 0.0) sincos(k * r, &sn, &cs);
        const double s4 = r > 0.0 ? 1.0 / (4.0 * PI * r) : 0.0;
        g[e] = mk<T>((T)(cs * s4), (T)(-sn * s4));
    }
}

LfArgs lf_args(pim_plan P, const LfGeom& G) {
    const PointsData& d = P->pts;
    LfArgs a{};
    a.lfslot = d.lfslot;
    a.segptr = d.segptr;
    a.seg = d.seg;
    a.lfself = d.lfself;
    a.lfnear = d.lfnear;
    a.lfl = d.lfl;
    a.bstart = d.bstart;
    a.blist = d.blist;
    a.dix = d.dix;
    a.lfp = d.lfp;
    a.pos = d.pos;
    a.nt = d.nt;
    a.ntd = d.ntd;
    a.perm = d.perm;
    a.phase = P->dphase;
    for (int i = 0; i < 3; ++i) {
        a.nb[i] = P->nb[i];
        a.nL[i] = P->n[i] - 1;
        a.n[i] = P->n[i];
        a.h[i] = P->h[i];
        a.D[i] = P->D[i];
        a.hf[i] = (float)P->h[i];
    }
    a.p = P->p;
    a.c = G.c;
    a.R = G.R;
    a.E = G.E;
    a.H = G.H;
    a.nimg = P->nimg;
    a.self_img = -1;
    for (int i = 0; i < P->nimg; ++i) {
        for (int k = 0; k < 3; ++k) a.img[i][k] = P->img[i][k];
        if (P->img[i][0] == 0 && P->img[i][1] == 0 && P->img[i][2] == 0) a.self_img = i;
    }
    a.k = P->k;
    // cos(k r) / (4 pi) = sum_t (-k^2)^t s^t / ((2t)! 4 pi),
    // -k sinc(k r) / (4 pi) = -k sum_t (-k^2)^t s^t / ((2t+1)! 4 pi)
    double f2 = 1.0, f1 = 1.0, pw = 1.0;
    for (int t = 0; t < LF_MAXNT; ++t) {
        if (t > 0) {
            f2 *= (2.0 * t - 1.0) * (2.0 * t);
            f1 *= (2.0 * t) * (2.0 * t + 1.0);
            pw *= -P->k * P->k;
        }
        a.pc[t] = (float)(pw / f2 / (4.0 * PI));
        a.ps[t] = (float)(-P->k * pw / f1 / (4.0 * PI));
    }
    a.nlf = d.nlf;
    a.status = P->dstatus;
    a.next = P->lfnext;
    return a;
}

// shared memory of the exact-part kernels (the point indices only in check
// mode, so that three FP32 CTAs fit an SM)
size_t lf_exact_smem(bool f64, bool check, bool sym = false) {
    const size_t segs = LF_MAXSEG * (sizeof(int4) + sizeof(int));
    if (f64) return LF_CH * (sizeof(dpos4) + sizeof(double2) + sizeof(int)) + segs;
    if (sym)
        return 1280 * (sizeof(float4) + sizeof(float2) + sizeof(int) + sizeof(float2)) +
               LF_MAXOBS * (2 * sizeof(float4) + 2 * sizeof(float) + sizeof(float2)) + segs;
    return LF_CH * (sizeof(float4) + sizeof(float2) + (check ? sizeof(int) : 0)) +
           LF_MAXOBS * (2 * sizeof(float4) + 2 * sizeof(float)) + segs;
}

template <typename T, int P>
size_t lf_grid_smem(const LfGeom& G) {
    constexpr int NP = P + 1;
    const size_t H1 = G.H + 1;
    return 2 * sizeof(T) * ((size_t)G.E * G.E * (G.EX + 1) + NP * NP * NP) + 32 + LF_MAXSLOT * sizeof(int2) +
           sizeof(int) * (3 * (size_t)G.E * G.E + 1) + (sizeof(T) == 4 ? sizeof(cplx<T>) * H1 * H1 * H1 : 0);
}

template <typename K>
pim_status set_smem(K kern, size_t bytes) {
    PIM_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return PIM_OK;
}

int lf_grid_blocks(long long nlf) { return (int)std::min<long long>(nlf, 152LL * 64); }

// resident CTAs of the exact-part kernel per SM: alone, as many as fit; on
// its own stream next to the spread, FFT and gather, one
constexpr int LF_CTAS_ALONE = 3, LF_CTAS_SHARED = 3;

template <int MODE>
pim_status launch_exact_f32(const LfGeom& G, const LfArgs& a, const void* qs, void* dst, cudaStream_t s,
                            int ctas_per_sm = LF_CTAS_ALONE, bool sym = false) {
    const size_t sm = lf_exact_smem(false, MODE == 2, sym && MODE != 2);
    const int nb = (int)std::min<long long>(a.nlf, 152LL * ctas_per_sm);
    PIM_CK(cudaMemsetAsync(a.next, 0, sizeof(unsigned long long), s));
    pim_status st;
#define PIM_LF_EX(NTV)                                                                              \
    do {                                                                                            \
        if (sym && MODE != 2) {                                                                     \
            if ((st = set_smem(lf_exact_f32<MODE, NTV, true>, sm)) != PIM_OK) return st;            \
            lf_exact_f32<MODE, NTV, true><<<nb, LF_NT, sm, s>>>(a, (const float2*)qs, dst);         \
        } else {                                                                                    \
            if ((st = set_smem(lf_exact_f32<MODE, NTV>, sm)) != PIM_OK) return st;                  \
            lf_exact_f32<MODE, NTV><<<nb, LF_NT, sm, s>>>(a, (const float2*)qs, dst);               \
        }                                                                                           \
    } while (0)
    if (MODE == 2 || G.nterm == 0) PIM_LF_EX(0);
    else if (G.nterm <= 4) PIM_LF_EX(4);
    else if (G.nterm <= 6) PIM_LF_EX(6);
    else PIM_LF_EX(8);
#undef PIM_LF_EX
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <int MODE>
pim_status launch_exact_f64(const LfArgs& a, const void* qs, void* dst, cudaStream_t s) {
    const size_t sm = lf_exact_smem(true, MODE == 2);
    pim_status st;
    if ((st = set_smem(lf_exact_f64<MODE>, sm)) != PIM_OK) return st;
    lf_exact_f64<MODE><<<lf_grid_blocks(a.nlf), LF_NT, sm, s>>>(a, (const double2*)qs, dst);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <typename T, int P, int EX>
pim_status launch_grid(const LfGeom& G, const LfArgs& a, bool adj, const void* qs, const void* mom, const void* gtab,
                       void* dst, cudaStream_t s) {
    const size_t sm = lf_grid_smem<T, P>(G);
    pim_status st;
    if (adj) {
        if ((st = set_smem(lf_grid_kernel<T, P, EX, true>, sm)) != PIM_OK) return st;
        lf_grid_kernel<T, P, EX, true><<<lf_grid_blocks(a.nlf), LF_GNT, sm, s>>>(a, (const cplx<T>*)mom,
                                                                                  (const cplx<T>*)gtab, dst);
    } else {
        if ((st = set_smem(lf_grid_kernel<T, P, EX, false>, sm)) != PIM_OK) return st;
        lf_grid_kernel<T, P, EX, false><<<lf_grid_blocks(a.nlf), LF_GNT, sm, s>>>(a, (const cplx<T>*)mom,
                                                                                   (const cplx<T>*)gtab, dst);
    }
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <typename T, int P>
pim_status launch_grid_p(const LfGeom& G, const LfArgs& a, bool adj, const void* qs, const void* mom,
                         const void* gtab, void* dst, cudaStream_t s) {
    if (G.EX == 16) return launch_grid<T, P, 16>(G, a, adj, qs, mom, gtab, dst, s);
    return launch_grid<T, P, 24>(G, a, adj, qs, mom, gtab, dst, s);
}

template <typename T>
pim_status launch_grid_t(const LfGeom& G, const LfArgs& a, bool adj, const void* qs, const void* mom,
                         const void* gtab, void* dst, cudaStream_t s) {
    switch (a.p) {
        case 2: return launch_grid_p<T, 2>(G, a, adj, qs, mom, gtab, dst, s);
        case 3: return launch_grid_p<T, 3>(G, a, adj, qs, mom, gtab, dst, s);
        default: return launch_grid_p<T, 4>(G, a, adj, qs, mom, gtab, dst, s);
    }
}

// the Q-output form of the grid kernel for `rows` boxes (FP32 plans)
template <int P, int EX>
pim_status launch_grid_q(const LfGeom& G, const LfArgs& a, bool adj, const void* mom, float* outh, long long rows,
                         cudaStream_t s) {
    // no kernel table in this form: two CTAs per SM where the full form has one
    const size_t H1 = G.H + 1;
    const size_t sm = lf_grid_smem<float, P>(G) - sizeof(float2) * H1 * H1 * H1;
    const int nb = (int)std::min<long long>(rows, 152LL * 64);
    pim_status st;
    if (adj) {
        if ((st = set_smem(lf_grid_kernel<float, P, EX, true, true>, sm)) != PIM_OK) return st;
        lf_grid_kernel<float, P, EX, true, true><<<nb, LF_GNT, sm, s>>>(a, (const float2*)mom, nullptr, outh);
    } else {
        if ((st = set_smem(lf_grid_kernel<float, P, EX, false, true>, sm)) != PIM_OK) return st;
        lf_grid_kernel<float, P, EX, false, true><<<nb, LF_GNT, sm, s>>>(a, (const float2*)mom, nullptr, outh);
    }
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <int P>
pim_status launch_grid_q_p(const LfGeom& G, const LfArgs& a, bool adj, const void* mom, float* outh, long long rows,
                           cudaStream_t s) {
    if (G.EX == 16) return launch_grid_q<P, 16>(G, a, adj, mom, outh, rows, s);
    return launch_grid_q<P, 24>(G, a, adj, mom, outh, rows, s);
}

// The tensor-core form of the grid part for the interior boxes, batch by
// batch: their local grids (Q rows), the product with the operator, and
// step 4 (out -= w . V, out in the layout LfArgs a describes).
pim_status lf_tc_run(pim_plan P, const LfGeom& G, const LfArgs& a, bool adj, void* out, cudaStream_t s) {
    const PointsData& d = P->pts;
    const long long K2 = 2LL * d.tcKP;
    const float* Ah = d.tcA + (adj ? 2 : 0) * (size_t)TC_M * K2;
    const float* Al = Ah + (size_t)TC_M * K2;
    float* Bq = d.tcB;
    pim_status st;
    if ((st = set_smem(lf_tc_gemm_kernel, TC_SMEM)) != PIM_OK) return st;
    for (long long b0 = 0; b0 < d.ntc; b0 += d.tcbatch) {
        const long long rows = std::min<long long>(d.tcbatch, d.ntc - b0);
        LfArgs q = a;
        q.tcl = d.tcl + b0;
        q.tcrows = rows;
        q.tcKP = d.tcKP;
        switch (P->p) {
            case 2: st = launch_grid_q_p<2>(G, q, adj, d.mom, Bq, rows, s); break;
            case 3: st = launch_grid_q_p<3>(G, q, adj, d.mom, Bq, rows, s); break;
            default: st = launch_grid_q_p<4>(G, q, adj, d.mom, Bq, rows, s); break;
        }
        if (st != PIM_OK) return st;
        if (b0 == 0) prof_mark(P, PIM_STAGE_LF_TC_GEMM, 0, s);
        lf_tc_gemm_kernel<<<(unsigned)((rows + TC_N - 1) / TC_N), TC_NT, TC_SMEM, s>>>(Ah, Al, Bq, (int)K2, rows, d.tcC,
                                                                                        a.status);
        PIM_CK(cudaGetLastError());
        if (b0 + rows >= d.ntc) prof_mark(P, PIM_STAGE_LF_TC_GEMM, 1, s);
        const unsigned nb = (unsigned)std::min<long long>((rows + 7) / 8, 152 * 16);
        switch (P->p) {
            case 2: lf_tc_interp_kernel<2><<<nb, 256, 0, s>>>(a, d.tcl + b0, rows, d.tcC, out); break;
            case 3: lf_tc_interp_kernel<3><<<nb, 256, 0, s>>>(a, d.tcl + b0, rows, d.tcC, out); break;
            default: lf_tc_interp_kernel<4><<<nb, 256, 0, s>>>(a, d.tcl + b0, rows, d.tcC, out); break;
        }
        PIM_CK(cudaGetLastError());
        P->launches += 3;
    }
    return PIM_OK;
}

}  // namespace

void lf_tc_free(pim_plan P) {
    PointsData& d = P->pts;
    const size_t K2 = 2 * (size_t)d.tcKP;
    pim_free(P, d.tcmask, d.tcmask ? (size_t)d.nlf : 0);
    pim_free(P, d.tcl, d.tcl ? (size_t)d.nlf * sizeof(int) : 0);
    pim_free(P, d.tcA, d.tcA ? 4 * (size_t)TC_M * K2 * sizeof(float) : 0);
    pim_free(P, d.tcB, d.tcB ? (size_t)d.tcbatch * K2 * sizeof(float) : 0);
    pim_free(P, d.tcC, d.tcC ? (size_t)d.tcbatch * TC_M * sizeof(float) : 0);
    d.tcmask = nullptr;
    d.tcl = nullptr;
    d.tcA = d.tcB = d.tcC = nullptr;
    d.ntc = 0;
    d.tcKP = 0;
    d.tcbatch = 0;
}

// The interior list-free boxes of an FP32 plan and the tables of their
// tensor-core grid part (after the list-free tables are built and nlf set).
pim_status lf_tc_prepare(pim_plan P, cudaStream_t s) {
    PointsData& d = P->pts;
    lf_tc_free(P);
    const LfGeom G = lf_geom(P);
    if (!P->lf_tc || P->prec != PIM_FP32_MIXED || d.nlf == 0 || G.EX == 0 || P->p < 2 || P->p > 4) return PIM_OK;
    pim_status st;
    int* cnt = nullptr;
    if ((st = pim_alloc(P, (void**)&d.tcmask, (size_t)d.nlf)) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.tcl, (size_t)d.nlf * sizeof(int))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&cnt, sizeof(int))) != PIM_OK) return st;
    PIM_CK(cudaMemsetAsync(cnt, 0, sizeof(int), s));
    const unsigned nb = (unsigned)std::min<long long>((d.nlf + 255) / 256, 152 * 16);
    lf_tc_list_kernel<<<nb, 256, 0, s>>>(d.lfslot, d.blist, d.segptr, d.nlf, P->nb[0], P->nb[1], P->n[0], P->n[1], P->n[2],
                                         G.c, P->p, G.R + G.c, G.R, d.tcmask, d.tcl, cnt);
    PIM_CK(cudaGetLastError());
    int ntc = 0;
    PIM_CK(cudaMemcpyAsync(&ntc, cnt, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, cnt, sizeof(int));
    d.ntc = ntc;
    if (ntc == 0) return PIM_OK;
    d.tcKP = (G.E * G.E * G.E + TC_K - 1) / TC_K * TC_K;
    const size_t K2 = 2 * (size_t)d.tcKP;
    d.tcbatch = std::min<long long>((ntc + TC_N - 1) / TC_N * TC_N, TC_BATCH);
    if ((st = pim_alloc(P, (void**)&d.tcA, 4 * (size_t)TC_M * K2 * sizeof(float))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.tcB, (size_t)d.tcbatch * K2 * sizeof(float))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.tcC, (size_t)d.tcbatch * TC_M * sizeof(float))) != PIM_OK) return st;
    const size_t A1 = (size_t)TC_M * K2;
    lf_tc_table_kernel<<<1024, 256, 0, s>>>(d.tcA, d.tcA + A1, d.tcA + 2 * A1, d.tcA + 3 * A1, G.E, d.tcKP, G.R + G.c,
                                            P->p + 1, P->h[0], P->h[1], P->h[2], P->k);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

LfGeom lf_geom(const pim_plan_s* P) {
    LfGeom G{};
    G.c = P->p / 2;
    G.R = P->b + 1;
    G.E = 2 * G.R + 2 * G.c + P->p + 1;
    G.H = G.R + 2 * G.c + P->p;
    G.EX = G.E <= 16 ? 16 : (G.E <= 24 ? 24 : 0);
    // the largest k r between an observer of a box and a point of its region:
    // box offsets up to R per axis plus half a box on each side
    double r2 = 0.0;
    for (int d = 0; d < 3; ++d) r2 += ((G.R + 1) * P->h[d]) * ((G.R + 1) * P->h[d]);
    const double x = P->k * std::sqrt(r2);
    // truncation of the cos series after t terms: x^(2t) / (2t)! (sinc: smaller)
    G.nterm = 0;
    double term = 1.0;
    for (int t = 1; t <= LF_MAXNT; ++t) {
        term *= x * x / ((2.0 * t - 1.0) * (2.0 * t));
        if (term < 1.5e-8) {
            G.nterm = std::max(t, 2);
            break;
        }
    }
    if (P->k == 0.0) G.nterm = 2;
    if (G.EX) {
        // the grid part's shared memory must fit one CTA
        const size_t NP = P->p + 1, H1 = G.H + 1;
        const size_t ts = P->prec == PIM_FP64 ? 8 : 4;
        const size_t sm = 2 * ts * ((size_t)G.E * G.E * (G.EX + 1) + NP * NP * NP) + 32 + 1024 * 8 +
                          4 * (3 * (size_t)G.E * G.E + 1) + (ts == 4 ? 8 * H1 * H1 * H1 : 0);
        if (sm > 227 * 1024) G.EX = 0;
    }
    return G;
}

pim_status lf_build_table(pim_plan P, cudaStream_t s) {
    PointsData& d = P->pts;
    const LfGeom G = lf_geom(P);
    const size_t H1 = G.H + 1;
    const size_t bytes = H1 * H1 * H1 * (P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2));
    pim_status st;
    if (!d.lfg && (st = pim_alloc(P, &d.lfg, bytes)) != PIM_OK) return st;
    if (P->prec == PIM_FP64)
        lf_table_kernel<double><<<64, 256, 0, s>>>((double2*)d.lfg, G.H, P->h[0], P->h[1], P->h[2], P->k);
    else
        lf_table_kernel<float><<<64, 256, 0, s>>>((float2*)d.lfg, G.H, P->h[0], P->h[1], P->h[2], P->k);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

// Flags pairs of list-free boxes that coincide (set-points check; the
// stored list checks its own pairs when it computes their values).
pim_status lf_check(pim_plan P, cudaStream_t s) {
    if (P->pts.nlf == 0) return PIM_OK;
    const LfGeom G = lf_geom(P);
    const LfArgs a = lf_args(P, G);
    if (P->prec == PIM_FP64) return launch_exact_f64<2>(a, nullptr, nullptr, s);
    return launch_exact_f32<2>(G, a, nullptr, nullptr, s);
}

// The list-free boxes' exact part into P->ulf (sorted order), on stream s:
// it reads only the sorted sources, so it runs while the spread, FFT and
// gather of the same apply run on the main stream.
pim_status lf_exact_async(pim_plan P, const void* qs, bool adj, cudaStream_t s) {
    if (P->pts.nlf == 0) return PIM_OK;
    const LfGeom G = lf_geom(P);
    LfArgs a = lf_args(P, G);
    if (adj) a.phase = P->dphase_adj;
    a.ulf = P->ulf;
    a.next = P->lfnext + pim_plan_s::RHS_LANES;  // its own box counter
    pim_status st;
    prof_mark(P, PIM_STAGE_LF_EXACT, 0, s);
    const bool sym = P->prec != PIM_FP64 && P->pts.xseg;
    if (sym) {
        // the pairs of two list-free boxes once for both (atomics into a zero ulf)
        a.seg = P->pts.xseg;
        a.segptr = P->pts.xsegptr;
        PIM_CK(cudaMemsetAsync(P->ulf, 0, (size_t)P->pts.N * sizeof(float2), s));
    }
    if (P->prec == PIM_FP64) st = adj ? launch_exact_f64<1>(a, qs, nullptr, s) : launch_exact_f64<0>(a, qs, nullptr, s);
    else
        st = adj ? launch_exact_f32<1>(G, a, qs, nullptr, s, LF_CTAS_SHARED, sym)
                 : launch_exact_f32<0>(G, a, qs, nullptr, s, LF_CTAS_SHARED, sym);
    prof_mark(P, PIM_STAGE_LF_EXACT, 1, s);
    P->launches += 1;
    return st;
}

// After lf_exact_async on the same stream and the spread of the same apply
// (the box moments): ulf -= the grid part, so that the whole list-free
// correction is formed off the main stream while the FFT and gather run.
pim_status lf_grid_async(pim_plan P, const void* qs, bool adj, cudaStream_t s) {
    if (P->pts.nlf == 0) return PIM_OK;
    const LfGeom G = lf_geom(P);
    LfArgs a = lf_args(P, G);
    if (adj) a.phase = P->dphase_adj;
    a.sorted_out = 1;  // into ulf, sorted order
    pim_status st;
    prof_mark(P, PIM_STAGE_LF_GRID, 0, s);
    if (P->pts.ntc > 0) {
        // the interior boxes on the tensor cores, the others below
        if ((st = lf_tc_run(P, G, a, adj, P->ulf, s)) != PIM_OK) return st;
        a.tcmask = P->pts.tcmask;
    }
    if (P->prec == PIM_FP64) st = launch_grid_t<double>(G, a, adj, qs, P->pts.mom, P->pts.lfg, P->ulf, s);
    else st = launch_grid_t<float>(G, a, adj, qs, P->pts.mom, P->pts.lfg, P->ulf, s);
    prof_mark(P, PIM_STAGE_LF_GRID, 1, s);
    P->launches += 1;
    return st;
}

// After lf_grid_async and the gather: dst += ulf for the list-free points.
pim_status lf_add(pim_plan P, void* dst, bool sorted_out, cudaStream_t s) {
    if (P->pts.nlf == 0) return PIM_OK;
    const LfGeom G = lf_geom(P);
    LfArgs a = lf_args(P, G);
    a.nrhs = 1;  // the concurrent form serves single right-hand sides
    a.r = 0;
    a.real_out = P->real_data && !sorted_out ? 1 : 0;
    a.sorted_out = sorted_out ? 1 : 0;
    const unsigned nb = (unsigned)std::min<long long>((P->pts.nlf + 7) / 8, 152 * 16);
    if (P->prec == PIM_FP64) lf_add_kernel<double><<<nb, 256, 0, s>>>(a, (const double2*)P->ulf, dst);
    else lf_add_kernel<float><<<nb, 256, 0, s>>>(a, (const float2*)P->ulf, dst);
    PIM_CK(cudaGetLastError());
    P->launches += 1;
    return PIM_OK;
}

// Adds the list-free boxes' corrections to the apply's output: the exact
// part, then minus the grid part (both read-modify-write dst after the
// gather has written it).  qs: sorted sources of right-hand side r.
pim_status lf_apply(pim_plan P, const void* qs, void* dst, int nrhs, int r, bool adj, bool sorted_out,
                    cudaStream_t s, int lane) {
    if (P->pts.nlf == 0) return PIM_OK;
    const LfGeom G = lf_geom(P);
    LfArgs a = lf_args(P, G);
    if (adj) a.phase = P->dphase_adj;
    a.next = P->lfnext + lane;  // the right-hand-side lanes run at once: a box counter each
    a.nrhs = nrhs;
    a.r = r;
    a.real_out = P->real_data && !sorted_out ? 1 : 0;
    a.sorted_out = sorted_out ? 1 : 0;
    pim_status st;
    prof_mark(P, PIM_STAGE_LF_EXACT, 0, s);
    if (P->prec == PIM_FP64) st = adj ? launch_exact_f64<1>(a, qs, dst, s) : launch_exact_f64<0>(a, qs, dst, s);
    else st = adj ? launch_exact_f32<1>(G, a, qs, dst, s) : launch_exact_f32<0>(G, a, qs, dst, s);
    if (st != PIM_OK) return st;
    prof_mark(P, PIM_STAGE_LF_EXACT, 1, s);
    prof_mark(P, PIM_STAGE_LF_GRID, 0, s);
    if (P->prec == PIM_FP64) st = launch_grid_t<double>(G, a, adj, qs, P->pts.mom, P->pts.lfg, dst, s);
    else st = launch_grid_t<float>(G, a, adj, qs, P->pts.mom, P->pts.lfg, dst, s);
    prof_mark(P, PIM_STAGE_LF_GRID, 1, s);
    P->launches += 2;
    return st;
}
