// The apply u = A q and its adjoint (Sec. 3.2 steps 1-3, Sec. 3.3 steps 1-4).
#include <algorithm>
#include <cmath>

#include "gather.cuh"
#include "lagrange.cuh"
#include "pim_internal.cuh"

namespace {

using namespace pim_k;

// ------------------------------- reductions --------------------------------
constexpr int RED_NT = 256, RED_BLOCKS = PIM_RED_BLOCKS;

template <typename T, bool REAL>
__device__ __forceinline__ double2 load_val(const void* q, long long i) {
    if (REAL) return make_double2((double)((const T*)q)[i], 0.0);
    const cplx<T> v = ((const cplx<T>*)q)[i];
    return make_double2((double)v.x, (double)v.y);
}

// partial[b] = (sum re, sum im, sum |q|) over a grid-stride slice, FP64
template <typename T, bool REAL>
__global__ void sum_partials_kernel(const void* q, long long N, int nrhs, int r, double* partial) {
    __shared__ double sh[3][RED_NT];
    double a = 0, b = 0, c = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const double2 v = load_val<T, REAL>(q, i * nrhs + r);
        a += v.x;
        b += v.y;
        c += sqrt(v.x * v.x + v.y * v.y);
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int s = RED_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) partial[3 * blockIdx.x + k] = sh[k][0];
}

// out = (mean re, mean im); raises the not-neutral flag if check and
// |sum q| > tol * sum |q| (Eq. neutral)
__global__ void sum_final_kernel(const double* partial, int nb, long long N, double tol, int check, double* out,
                                 int* status) {
    __shared__ double sh[3][RED_NT];
    double a = 0, b = 0, c = 0;
    for (int i = threadIdx.x; i < nb; i += RED_NT) {
        a += partial[3 * i];
        b += partial[3 * i + 1];
        c += partial[3 * i + 2];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int s = RED_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sh[0][0] / (double)N;
        out[1] = sh[1][0] / (double)N;
        if (check && sqrt(sh[0][0] * sh[0][0] + sh[1][0] * sh[1][0]) > tol * sh[2][0]) atomicOr(status, PIM_DEV_NOT_NEUTRAL);
    }
}

// qs[m] = q[perm[m]] - mean (sorted order, plan precision)
template <typename T, bool REAL>
__global__ void permute_kernel(const void* q, const int* perm, long long N, int nrhs, int r, const double* mean,
                               cplx<T>* qs) {
    const double mr = mean ? mean[0] : 0.0, mi = mean ? mean[1] : 0.0;
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const double2 v = load_val<T, REAL>(q, (long long)perm[m] * nrhs + r);
        qs[m] = mk<T>((T)(v.x - mr), (T)(v.y - mi));
    }
}

// ------------------------------- near spread -------------------------------


// Q(a) = sum_n w_n(a) q_n (Sec. 3.3 step 1) without global atomics.
// Every point of a box shares the box's stencil start s_b, so the points of
// a box with many points are first summed into the box's (p+1)^3 moments
//   M_b(j) = sum_{n in b} w_n(j) q_n,        Q(a) = sum_b M_b(a - s_b),
// while the points of the other boxes are added one by one.  Phase 1 forms
// the moments of the dense boxes; phase 2 builds every grid line (y, z) in
// shared memory from the "entries" (a dense box or a single point) of the box
// rows whose stencils cover the line.
template <int P>
__device__ __forceinline__ void covering_boxes(int a, int n, int nb, int& lo, int& hi) {
    constexpr int LO = (P & 1) ? (P - 1) / 2 : P / 2;
    lo = a <= P ? 0 : a - P + LO;
    hi = a >= n - 1 - P ? nb - 1 : a + LO;
    lo = max(lo, 0);
    hi = min(hi, nb - 1);
}

struct MomentArgs {
    long long nd;
    const int* dslot;    // slot of each dense box
    const int* bstart;   // nne + 1 point offsets of the non-empty boxes
    const float* nt;
    const double* ntd;
};

// Phase 1: one warp per dense box.  Lane l < (P+1)^2 owns the stencil
// offsets (jx = 0..P, jy = l % (P+1), jz = l / (P+1)); the box's points are
// loaded 32 at a time and walked by shuffles; for each point, lane l < 3(P+1)
// evaluates the one weight w_{l % (P+1)} along axis l / (P+1) and the others
// fetch it.  The row of moments is written once (lane l: P+1 consecutive
// values, the warp one contiguous row).
template <typename T, int P>
__global__ void __launch_bounds__(256) moment_kernel(MomentArgs a, const cplx<T>* __restrict__ qs, cplx<T>* mom) {
    constexpr int NP = P + 1, NP3 = NP * NP * NP;
    static_assert(NP * NP <= 32, "one lane per (jy, jz) pair");
    const int lane = threadIdx.x & 31;
    const long long dbox = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (dbox >= a.nd) return;
    const int jy = lane % NP, jz = lane / NP;
    const int wd = min(lane / NP, 2), wj = lane % NP;  // the weight this lane evaluates
    const int slot = a.dslot[dbox];
    const int m0 = a.bstart[slot], m1 = a.bstart[slot + 1];
    cplx<T> sum[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) sum[j] = mk<T>(T(0), T(0));
    for (int b0 = m0; b0 < m1; b0 += 32) {
        const int cnt = min(32, m1 - b0);
        const int ml = b0 + lane;
        T tl[3] = {T(0), T(0), T(0)};
        cplx<T> ql = mk<T>(T(0), T(0));
        if (lane < cnt) {
#pragma unroll
            for (int d = 0; d < 3; ++d) tl[d] = sizeof(T) == 8 ? (T)a.ntd[3 * ml + d] : (T)a.nt[3 * ml + d];
            ql = qs[ml];
        }
        for (int j = 0; j < cnt; ++j) {
            const T tx = __shfl_sync(0xffffffffu, tl[0], j), ty = __shfl_sync(0xffffffffu, tl[1], j),
                    tz = __shfl_sync(0xffffffffu, tl[2], j);
            const T qx = __shfl_sync(0xffffffffu, ql.x, j), qy = __shfl_sync(0xffffffffu, ql.y, j);
            const T wl = lag1<T, P>(wd == 0 ? tx : (wd == 1 ? ty : tz), wj);
            T wx[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) wx[i] = __shfl_sync(0xffffffffu, wl, i);
            const T wyz = __shfl_sync(0xffffffffu, wl, NP + jy) * __shfl_sync(0xffffffffu, wl, 2 * NP + jz);
            const T cx = wyz * qx, cy = wyz * qy;
#pragma unroll
            for (int i = 0; i < NP; ++i) {
                sum[i].x += wx[i] * cx;
                sum[i].y += wx[i] * cy;
            }
        }
    }
    if (lane < NP * NP) {
        cplx<T>* out = mom + dbox * NP3 + lane * NP;
#pragma unroll
        for (int i = 0; i < NP; ++i) out[i] = sum[i];
    }
}

// Phase 2: one warp per grid line (y, z) along x, the line kept in shared
// memory.  The box rows whose stencils cover (y, z) (<= (P+1)^2 in the
// interior) go to lanes, and their entries are enumerated as one flat list
// (a warp prefix sum of the row counts), so that the loads of all rows are
// in flight together.  An entry adds P+1 values at x = s_x..s_x+P of the
// line: a dense box its moments M_b(0..P, jy, jz), a point
// w_x(0..P) w_y(jy) w_z(jz) q_n.
struct LineArgs {
    int n[3], nb[3];
    int ncopy;             // copies of the line in shared memory (1, 2 or 4)
    const int* eptr;       // first entry of each box row
    const uint32_t* ent;   // entries: dense box (bit 31 | dense index) or point
    const uint16_t* esx;   // stencil start along x of each entry
    const float* nt;
    const double* ntd;
};

// Shared-memory layout of one warp's line: ncopy copies, each a real and an
// imaginary array of line_ld(nx) words; copy c starts 8c words past a
// multiple of 32, so that equal x in different copies fall in different
// banks.  Consecutive box rows of a chunk add into different copies, so the
// atomics of one instruction rarely share an address.
__host__ __device__ __forceinline__ int line_ld(int nx) { return ((nx + 31) & ~31) + 16; }
__host__ __device__ __forceinline__ int line_words(int nx, int ncopy) { return ncopy * (2 * line_ld(nx) + 8); }

template <int P>
__device__ __forceinline__ int sclamp(int b, int n) {
    constexpr int LO = (P & 1) ? (P - 1) / 2 : P / 2;
    return min(max(b - LO, 0), n - 1 - P);
}

template <typename T, int P>
__global__ void __launch_bounds__(256) line_kernel(LineArgs a, const cplx<T>* __restrict__ mom,
                                                   const cplx<T>* __restrict__ qs, cplx<T>* Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NP = P + 1, NP3 = NP * NP * NP;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nx = a.n[0];
    const int ld = line_ld(nx), cw = 2 * ld + 8;
    T* L = reinterpret_cast<T*>(smem_raw) + (size_t)wid * line_words(nx, a.ncopy);
    const long long line = (long long)blockIdx.x * (blockDim.x >> 5) + wid;
    if (line >= (long long)a.n[1] * a.n[2]) return;
    const int y = (int)(line % a.n[1]), z = (int)(line / a.n[1]);
    for (int i = lane; i < line_words(nx, a.ncopy); i += 32) L[i] = T(0);
    __syncwarp();
    int ylo, yhi, zlo, zhi;
    covering_boxes<P>(y, a.n[1], a.nb[1], ylo, yhi);
    covering_boxes<P>(z, a.n[2], a.nb[2], zlo, zhi);
    const int nyc = yhi - ylo + 1, ncand = nyc * (zhi - zlo + 1);
    for (int c0 = 0; c0 < ncand; c0 += 32) {
        // lane: one candidate box row (by, bz) and its entry range
        const int c = c0 + lane;
        const int by = ylo + c % nyc, bz = zlo + c / nyc;
        const int jy = y - sclamp<P>(by, a.n[1]), jz = z - sclamp<P>(bz, a.n[2]);
        int s0 = 0, cnt = 0;
        if (c < ncand && (unsigned)jy <= (unsigned)P && (unsigned)jz <= (unsigned)P) {
            const long long r = (long long)bz * a.nb[1] + by;
            s0 = a.eptr[r];
            cnt = a.eptr[r + 1] - s0;
        }
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int excl = incl - cnt, total = __shfl_sync(0xffffffffu, incl, 31);
        const int jyz = jz * NP + jy;
        for (int t0 = 0; t0 < total; t0 += 64) {
            // two entries per lane, all loads issued before the adds
            int e[2], rjyz[2], cp[2];
            bool ok[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = t0 + 32 * h + lane;
                int k = 0;  // owner: the last lane whose range starts at or before t
#pragma unroll
                for (int st = 16; st > 0; st >>= 1) {
                    const int ex = __shfl_sync(0xffffffffu, excl, k + st);
                    if (ex <= t) k += st;
                }
                ok[h] = t < total;
                e[h] = __shfl_sync(0xffffffffu, s0, k) + (t - __shfl_sync(0xffffffffu, excl, k));
                rjyz[h] = __shfl_sync(0xffffffffu, jyz, k);
                cp[h] = (k % a.ncopy) * cw;
            }
            uint32_t desc[2];
            int sx[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                desc[h] = ok[h] ? a.ent[e[h]] : 0u;
                sx[h] = ok[h] ? (int)a.esx[e[h]] : 0;
            }
            cplx<T> v[2][NP];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (desc[h] & 0x80000000u) {
                    const cplx<T>* src = mom + (long long)(desc[h] & 0x7fffffffu) * NP3 + rjyz[h] * NP;
#pragma unroll
                    for (int j = 0; j < NP; ++j) v[h][j] = src[j];
                } else {
                    // a single point: w_x(0..P) w_y(jy) w_z(jz) q_n
                    const long long m = desc[h];
                    T t[3];
#pragma unroll
                    for (int d = 0; d < 3; ++d) t[d] = sizeof(T) == 8 ? (T)a.ntd[3 * m + d] : (T)a.nt[3 * m + d];
                    const cplx<T> q = ok[h] ? qs[m] : mk<T>(T(0), T(0));
                    T wx[NP];
                    lagrange_w<T, P>(t[0], wx);
                    const T wyz = lag1<T, P>(t[1], rjyz[h] % NP) * lag1<T, P>(t[2], rjyz[h] / NP);
                    const T cx = wyz * q.x, cy = wyz * q.y;
#pragma unroll
                    for (int j = 0; j < NP; ++j) v[h][j] = mk<T>(wx[j] * cx, wx[j] * cy);
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok[h]) continue;
                T* Lr = L + cp[h];
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    atomicAdd(Lr + sx[h] + j, v[h][j].x);
                    atomicAdd(Lr + ld + sx[h] + j, v[h][j].y);
                }
            }
        }
    }
    __syncwarp();
    cplx<T>* out = Q + ((long long)z * a.n[1] + y) * nx;
    for (int x = lane; x < nx; x += 32) {
        T re = L[x], im = L[ld + x];
        for (int c = 1; c < a.ncopy; ++c) {
            re += L[c * cw + x];
            im += L[c * cw + ld + x];
        }
        out[x] = mk<T>(re, im);
    }
}

template <typename T, int P>
pim_status spread_two_phase(pim_plan P_, const cplx<T>* qs, cplx<T>* Q, cudaStream_t s) {
    const PointsData& d = P_->pts;
    MomentArgs ma{};
    ma.nd = d.nd;
    ma.dslot = d.dslot;
    ma.bstart = d.bstart;
    ma.nt = d.nt;
    ma.ntd = d.ntd;
    if (d.nd > 0) moment_kernel<T, P><<<(unsigned)((d.nd * 32 + 255) / 256), 256, 0, s>>>(ma, qs, (cplx<T>*)d.mom);
    LineArgs la{};
    for (int i = 0; i < 3; ++i) { la.n[i] = P_->n[i]; la.nb[i] = P_->nb[i]; }
    la.eptr = d.eptr;
    la.ent = d.ent;
    la.esx = d.esx;
    la.nt = d.nt;
    la.ntd = d.ntd;
    const long long nlines = (long long)P_->n[1] * P_->n[2];
    // as many line copies as fit in 96 KB per CTA of 8 warps
    la.ncopy = 4;
    while (la.ncopy > 1 && 8 * sizeof(T) * (size_t)line_words(P_->n[0], la.ncopy) > 96 * 1024) la.ncopy /= 2;
    const size_t sm = 8 * sizeof(T) * (size_t)line_words(P_->n[0], la.ncopy);
    PIM_CK(cudaFuncSetAttribute(line_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    line_kernel<T, P><<<(unsigned)((nlines + 7) / 8), 256, sm, s>>>(la, (const cplx<T>*)d.mom, qs, Q);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

// ------------------------------- far spread --------------------------------
struct FarSpreadArgs {
    int nf[3], pf;
    long long N;
    int chunk;             // points per CTA
    const uint32_t* fst;   // stencil starts of the grid spread onto
    const float* ft;       // local coordinates (stride 6, offset toff)
    const double* ftd;
    int toff;
    const int* fperm;      // the points in order of their stencil start on that grid (or null: box order)
};

// Per-CTA partial far-grid charges (Eq. projection) in shared memory.  Each
// warp walks a contiguous run of (spatially sorted) points; lane (jy, jz)
// owns one x-row of the far stencil and keeps its P+1 sums in registers
// while consecutive points share a stencil start, adding them to shared
// memory when the start changes (the lanes of one flush write distinct
// rows, so their atomics do not collide).
//
// WIN: for far grids too large for a copy per CTA.  The CTA's points (a run
// of the box-sorted points, so a thin slab in z) have far stencils in a few
// consecutive z planes; the CTA accumulates those planes in shared memory
// and adds them to the FP64 far grid `grid` with atomics (a CTA whose planes
// do not fit in maxplanes adds its sums to `grid` directly).
template <typename T, int PF, bool WIN>
__global__ void __launch_bounds__(256) far_spread_kernel(FarSpreadArgs a, const cplx<T>* __restrict__ qs,
                                                         cplx<T>* part, double2* grid, int maxplanes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);
    __shared__ int zr[2];
    constexpr int NP = PF + 1, KP = (NP * NP + 31) / 32;  // (jy, jz) rows per lane
    static_assert(3 * NP <= 32, "one lane per weight");
    const int plane = a.nf[0] * a.nf[1];
    const long long m0 = (long long)blockIdx.x * a.chunk;
    const long long m1 = min(a.N, m0 + a.chunk);
    int G = a.nf[2] * plane, zoff = 0;
    bool inshared = true;
    if (WIN) {
        if (threadIdx.x == 0) {
            zr[0] = 1 << 30;
            zr[1] = -1;
        }
        __syncthreads();
        for (long long m = m0 + threadIdx.x; m < m1; m += blockDim.x) {
            const int z = (int)((a.fst[a.fperm ? a.fperm[m] : m] >> 20) & 1023);
            atomicMin(&zr[0], z);
            atomicMax(&zr[1], z);
        }
        __syncthreads();
        zoff = zr[0] * plane;
        G = (zr[1] - zr[0] + PF + 1) * plane;
        inshared = zr[1] >= zr[0] && zr[1] - zr[0] + PF + 1 <= maxplanes;
    }
    if (inshared)
        for (int i = threadIdx.x; i < 2 * G; i += blockDim.x) acc[i] = T(0);
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long per = (m1 - m0 + nw - 1) / nw;
    const long long w0 = m0 + wid * per, w1 = min(m1, w0 + per);
    const int wd = min(lane / NP, 2), wj = lane % NP;  // the weight this lane evaluates
    bool act[KP];
    int jy[KP], jz[KP], base[KP];
    cplx<T> sum[KP][NP];
#pragma unroll
    for (int k = 0; k < KP; ++k) {
        const int l = lane + 32 * k;
        act[k] = l < NP * NP;
        jy[k] = act[k] ? l % NP : 0;
        jz[k] = act[k] ? l / NP : 0;
        base[k] = 0;
#pragma unroll
        for (int i = 0; i < NP; ++i) sum[k][i] = mk<T>(T(0), T(0));
    }
    uint32_t cur = 0xffffffffu;
    auto flush = [&]() {
#pragma unroll
        for (int k = 0; k < KP; ++k)
            if (act[k]) {
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    if (inshared) {
                        atomicAdd(acc + 2 * (base[k] - zoff + i), sum[k][i].x);
                        atomicAdd(acc + 2 * (base[k] - zoff + i) + 1, sum[k][i].y);
                    } else {
                        atomicAdd(&grid[base[k] + i].x, (double)sum[k][i].x);
                        atomicAdd(&grid[base[k] + i].y, (double)sum[k][i].y);
                    }
                }
            }
    };
    for (long long b0 = w0; b0 < w1; b0 += 32) {
        const int cnt = (int)min(32LL, w1 - b0);
        const long long ml = b0 + lane;
        uint32_t sl = 0;
        T tl[3] = {T(0), T(0), T(0)};
        cplx<T> ql = mk<T>(T(0), T(0));
        if (lane < cnt) {
            const long long mm = a.fperm ? (long long)a.fperm[ml] : ml;
            sl = a.fst[mm];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                tl[d] = sizeof(T) == 8 ? (T)a.ftd[6 * mm + a.toff + d] : (T)a.ft[6 * mm + a.toff + d];
            ql = qs[mm];
        }
        for (int j = 0; j < cnt; ++j) {
            const uint32_t sm = __shfl_sync(0xffffffffu, sl, j);
            if (sm != cur) {
                if (cur != 0xffffffffu) flush();
                cur = sm;
                int s3[3];
                unpack3(sm, s3[0], s3[1], s3[2]);
#pragma unroll
                for (int k = 0; k < KP; ++k) {
                    base[k] = ((s3[2] + jz[k]) * a.nf[1] + (s3[1] + jy[k])) * a.nf[0] + s3[0];
#pragma unroll
                    for (int i = 0; i < NP; ++i) sum[k][i] = mk<T>(T(0), T(0));
                }
            }
            const T tx = __shfl_sync(0xffffffffu, tl[0], j), ty = __shfl_sync(0xffffffffu, tl[1], j),
                    tz = __shfl_sync(0xffffffffu, tl[2], j);
            const T qx = __shfl_sync(0xffffffffu, ql.x, j), qy = __shfl_sync(0xffffffffu, ql.y, j);
            // lane l < 3(P+1) evaluates the one weight w_{l % (P+1)} of axis
            // l / (P+1); every lane then fetches the weights it needs
            const T wl = lag1<T, PF>(wd == 0 ? tx : (wd == 1 ? ty : tz), wj);
            T wx[NP];
#pragma unroll
            for (int i = 0; i < NP; ++i) wx[i] = __shfl_sync(0xffffffffu, wl, i);
#pragma unroll
            for (int k = 0; k < KP; ++k) {
                const T wyz = __shfl_sync(0xffffffffu, wl, NP + jy[k]) * __shfl_sync(0xffffffffu, wl, 2 * NP + jz[k]);
                const T cx = wyz * qx, cy = wyz * qy;
#pragma unroll
                for (int i = 0; i < NP; ++i) {
                    sum[k][i].x += wx[i] * cx;
                    sum[k][i].y += wx[i] * cy;
                }
            }
        }
    }
    if (cur != 0xffffffffu) flush();
    __syncthreads();
    if (WIN) {
        if (inshared)
            for (int i = threadIdx.x; i < G; i += blockDim.x) {
                const T re = acc[2 * i], im = acc[2 * i + 1];
                if (re != T(0) || im != T(0)) {
                    atomicAdd(&grid[zoff + i].x, (double)re);
                    atomicAdd(&grid[zoff + i].y, (double)im);
                }
            }
        return;
    }
    cplx<T>* out = part + (long long)blockIdx.x * G;
    for (int i = threadIdx.x; i < G; i += blockDim.x) out[i] = mk<T>(acc[2 * i], acc[2 * i + 1]);
}

template <typename T, bool WIN>
pim_status launch_far_spread_k(int pf, int grid, size_t sm, cudaStream_t s, const FarSpreadArgs& fa,
                               const cplx<T>* qs, cplx<T>* part, double2* out, int maxplanes) {
#define PIM_FAR_CASE(PFV)                                                                                         \
    case PFV: {                                                                                                   \
        PIM_CK(cudaFuncSetAttribute(far_spread_kernel<T, PFV, WIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    (int)sm));                                                                    \
        far_spread_kernel<T, PFV, WIN><<<grid, 256, sm, s>>>(fa, qs, part, out, maxplanes);                       \
        break;                                                                                                    \
    }
    switch (pf) {
        PIM_FAR_CASE(2)
        PIM_FAR_CASE(3)
        PIM_FAR_CASE(4)
        PIM_FAR_CASE(5)
        PIM_FAR_CASE(6)
        default: pim_set_error("far degree must be 2..6"); return PIM_ERR_UNSUPPORTED;
    }
#undef PIM_FAR_CASE
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

// qf[g] = sum over CTAs of the partials, in FP64, fixed order: one warp
// per far node, lanes stride the partials, then a shuffle tree.
template <typename T>
__global__ void far_reduce_kernel(const cplx<T>* part, int nchunks, int G, double2* qf) {
    const int lane = threadIdx.x & 31;
    const long long w0 = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long g = w0; g < G; g += nw) {
        double2 s = make_double2(0.0, 0.0);
        for (int c = lane; c < nchunks; c += 32) {
            const cplx<T> v = part[(long long)c * G + g];
            s.x += (double)v.x;
            s.y += (double)v.y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
        }
        if (lane == 0) qf[g] = s;
    }
}

// The far grid charges (Eq. projection) of the sorted sources into the FP64
// grid `out`: per-CTA partial grids in shared memory, reduced in a fixed
// order (far grids up to 200 KB of plan-precision complex values), or
// shared-memory z-windows added with FP64 atomics (larger far grids).
template <typename T>
pim_status far_spread_grid(pim_plan P, long long N, const uint32_t* fst, int toff, const cplx<T>* src,
                           double2* out, cudaStream_t s) {
    const PointsData& d = P->pts;
    const int G = P->nf[0] * P->nf[1] * P->nf[2];
    FarSpreadArgs fa{};
    for (int i = 0; i < 3; ++i) fa.nf[i] = P->nf[i];
    fa.pf = P->pf;
    fa.N = N;
    fa.fst = fst;
    fa.ft = d.ft;
    fa.ftd = d.ftd;
    fa.toff = toff;
    fa.fperm = fst == d.fs ? d.fperm_s : (fst == d.fo ? d.fperm_o : nullptr);
    pim_status st;
    if (!P->far_window) {
        fa.chunk = (int)((N + P->far_chunks - 1) / P->far_chunks);
        const size_t sm = 2 * sizeof(T) * G;
        if (N > 0) {
            if ((st = launch_far_spread_k<T, false>(P->pf, P->far_chunks, sm, s, fa, src, (cplx<T>*)P->fpart, nullptr,
                                                    0)) != PIM_OK)
                return st;
        } else {
            PIM_CK(cudaMemsetAsync(P->fpart, 0, sizeof(cplx<T>) * G * P->far_chunks, s));
        }
        far_reduce_kernel<T><<<(G * 32 + 255) / 256, 256, 0, s>>>((const cplx<T>*)P->fpart, P->far_chunks, G, out);
        PIM_CK(cudaGetLastError());
        P->launches += 2;
        return PIM_OK;
    }
    PIM_CK(cudaMemsetAsync(out, 0, sizeof(double2) * G, s));
    if (N == 0) return PIM_OK;
    const int plane = P->nf[0] * P->nf[1];
    const int maxplanes = (int)std::max<long long>(1, (200 * 1024) / (2 * sizeof(T) * (long long)plane));
    const int nchunk = (int)std::max<long long>(1, std::min<long long>(152LL * 8, (N + 2047) / 2048));
    fa.chunk = (int)((N + nchunk - 1) / nchunk);
    const size_t sm = 2 * sizeof(T) * (size_t)maxplanes * plane;
    if ((st = launch_far_spread_k<T, true>(P->pf, nchunk, sm, s, fa, src, nullptr, out, maxplanes)) != PIM_OK)
        return st;
    P->launches += 1;
    return PIM_OK;
}

// Far gather (Eq. interpolation) of every point into ufp, in the caller's
// order, one thread per point: its (PF+1)^3 observer-stencil weights once,
// then the stencil's x-rows of the far grid (small, cache-resident).  Runs on
// the far stream while the near gather runs on the main one.
template <typename T, int PF>
__global__ void __launch_bounds__(256) far_interp_kernel(GatherArgs a, const cplx<T>* __restrict__ uf,
                                                         cplx<T>* __restrict__ ufp) {
    constexpr int NP = PF + 1;
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (m >= a.N) return;
    int f[3];
    unpack3(a.fst[m], f[0], f[1], f[2]);
    T w[3][NP];
#pragma unroll
    for (int d = 0; d < 3; ++d)
        lagrange_w<T, PF>(sizeof(T) == 8 ? (T)a.ftd[6 * m + a.toff + d] : (T)a.ft[6 * m + a.toff + d], w[d]);
    cplx<T> acc = mk<T>(T(0), T(0));
#pragma unroll
    for (int jz = 0; jz < NP; ++jz) {
        cplx<T> az = mk<T>(T(0), T(0));
#pragma unroll
        for (int jy = 0; jy < NP; ++jy) {
            const cplx<T>* row = uf + ((long long)(f[2] + jz) * a.nf[1] + (f[1] + jy)) * a.nf[0] + f[0];
            cplx<T> r = mk<T>(T(0), T(0));
#pragma unroll
            for (int jx = 0; jx < NP; ++jx) {
                const cplx<T> v = __ldg(row + jx);
                r.x += w[0][jx] * v.x;
                r.y += w[0][jx] * v.y;
            }
            az.x += w[1][jy] * r.x;
            az.y += w[1][jy] * r.y;
        }
        acc.x += w[2][jz] * az.x;
        acc.y += w[2][jz] * az.y;
    }
    ufp[a.perm[m]] = acc;
}

template <typename T>
pim_status launch_far_interp(int pf, long long N, cudaStream_t s, const GatherArgs& fg, const cplx<T>* uf,
                             cplx<T>* ufp) {
    const unsigned nb = (unsigned)((N + 255) / 256);
    switch (pf) {
        case 2: far_interp_kernel<T, 2><<<nb, 256, 0, s>>>(fg, uf, ufp); break;
        case 3: far_interp_kernel<T, 3><<<nb, 256, 0, s>>>(fg, uf, ufp); break;
        case 4: far_interp_kernel<T, 4><<<nb, 256, 0, s>>>(fg, uf, ufp); break;
        case 5: far_interp_kernel<T, 5><<<nb, 256, 0, s>>>(fg, uf, ufp); break;
        case 6: far_interp_kernel<T, 6><<<nb, 256, 0, s>>>(fg, uf, ufp); break;
        default: pim_set_error("far degree must be 2..6"); return PIM_ERR_UNSUPPORTED;
    }
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

// u += far part (Eq. 5's near and far zones summed, after both streams have
// joined): coalesced in the caller's order, or gathered for the sorted output
// of the neutral-static adjoint.
template <typename T>
__global__ void far_add_kernel(GatherArgs a, const cplx<T>* __restrict__ ufp, void* out) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < a.N;
         i += (long long)gridDim.x * blockDim.x) {
        if (a.sorted_out) {
            const cplx<T> f = ufp[a.perm[i]];
            cplx<T>* u = (cplx<T>*)out + i;
            *u = mk<T>(u->x + f.x, u->y + f.y);
        } else {
            const cplx<T> f = ufp[i];
            const long long o = i * a.nrhs + a.r;
            if (a.real_out) {
                ((T*)out)[o] += f.x;
            } else {
                cplx<T>* u = (cplx<T>*)out + o;
                *u = mk<T>(u->x + f.x, u->y + f.y);
            }
        }
    }
}

template <typename T>
__global__ void far_convert_kernel(const double2* in, cplx<T>* out, int G) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G; g += gridDim.x * blockDim.x)
        out[g] = mk<T>((T)in[g].x, (T)in[g].y);
}

// ------------------------------- position gradient -------------------------
struct GradArgs {
    int n[3], nf[3], pf;
    const int* nbig;          // compact mode: the rows' double-float entries (else null: all of them)
    const float2* dvalf;      // 3 per entry, FP32 heads of the derivatives (compact mode)
    double h[3], df[3];
    long long N;
    int has_far, self_img, first;
    const int* perm;
    const uint32_t* ns;
    const float* nt;
    const double* ntd;
    const uint32_t* fs;
    const uint32_t* fo;
    const float* ft;
    const double* ftd;
    const int64_t* row_ptr;
    const uint32_t* col;
    const double2* dval;      // 3 per entry, FP64
    const float4* dvaldf;     // 3 per entry, double-float (double-float correction mode)
    const double2* phase;
    const float4* phasedf;
};

// One stencil's contribution to a point's gradient, lane (jy, jz) taking
// the x-row: adds Re[conj(g_k) (grad w . U)] + Re[q_k conj(grad w . V)] to
// part[0..2], with the weights of degree PF (compile time) at local
// coordinates t (grid steps) and 1/h the inverse spacings.
template <typename T, int PF>
__device__ __forceinline__ void grad_stencil(const T* t, const double* h, int jy, int jz, const cplx<T>* rowU,
                                             const cplx<T>* rowV, cplx<T> gm, cplx<T> qm, T* part) {
    constexpr int NP = PF + 1;
    T w[3][NP], dw[3][NP];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lagrange_wdw<T, PF>(t[d], w[d], dw[d]);
        const T ih = T(1.0 / h[d]);
#pragma unroll
        for (int j = 0; j < NP; ++j) dw[d][j] *= ih;
    }
    const T wy = pick<NP>(w[1], jy), dwy = pick<NP>(dw[1], jy);
    const T wz = pick<NP>(w[2], jz), dwz = pick<NP>(dw[2], jz);
    // A = sum w'_x U, B = sum w_x U (C, D the same for V); the row adds
    // (w_y w_z A, w'_y w_z B, w_y w'_z B) to the three gradient components
    cplx<T> A = mk<T>(T(0), T(0)), B = A, C = A, D = A;
#pragma unroll
    for (int jx = 0; jx < NP; ++jx) {
        if (rowU) {
            const cplx<T> u = rowU[jx];
            A.x += dw[0][jx] * u.x; A.y += dw[0][jx] * u.y;
            B.x += w[0][jx] * u.x;  B.y += w[0][jx] * u.y;
        }
        if (rowV) {
            const cplx<T> v = rowV[jx];
            C.x += dw[0][jx] * v.x; C.y += dw[0][jx] * v.y;
            D.x += w[0][jx] * v.x;  D.y += w[0][jx] * v.y;
        }
    }
    // Re[conj(g) X] = g.x X.x + g.y X.y and Re[q conj(Y)] = q.x Y.x + q.y Y.y
    const T ra = gm.x * A.x + gm.y * A.y + qm.x * C.x + qm.y * C.y;
    const T rb = gm.x * B.x + gm.y * B.y + qm.x * D.x + qm.y * D.y;
    part[0] += wy * wz * ra;
    part[1] += dwy * wz * rb;
    part[2] += wy * dwz * rb;
}

// The same for a runtime far degree p <= PIM_MAX_P.
template <typename T>
__device__ __forceinline__ void grad_stencil_rt(int p, const T* t, const double* h, int jy, int jz,
                                                const cplx<T>* rowU, const cplx<T>* rowV, cplx<T> gm, cplx<T> qm,
                                                T* part) {
    T w[3][PIM_MAX_P + 1], dw[3][PIM_MAX_P + 1];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lagrange_wdw_rt<T>(p, t[d], w[d], dw[d]);
        const T ih = T(1.0 / h[d]);
#pragma unroll
        for (int j = 0; j <= PIM_MAX_P; ++j) dw[d][j] *= ih;
    }
    const T wy = pick<PIM_MAX_P + 1>(w[1], jy), dwy = pick<PIM_MAX_P + 1>(dw[1], jy);
    const T wz = pick<PIM_MAX_P + 1>(w[2], jz), dwz = pick<PIM_MAX_P + 1>(dw[2], jz);
    cplx<T> A = mk<T>(T(0), T(0)), B = A, C = A, D = A;
#pragma unroll
    for (int jx = 0; jx <= PIM_MAX_P; ++jx) {
        if (jx > p) break;
        if (rowU) {
            const cplx<T> u = rowU[jx];
            A.x += dw[0][jx] * u.x; A.y += dw[0][jx] * u.y;
            B.x += w[0][jx] * u.x;  B.y += w[0][jx] * u.y;
        }
        if (rowV) {
            const cplx<T> v = rowV[jx];
            C.x += dw[0][jx] * v.x; C.y += dw[0][jx] * v.y;
            D.x += w[0][jx] * v.x;  D.y += w[0][jx] * v.y;
        }
    }
    const T ra = gm.x * A.x + gm.y * A.y + qm.x * C.x + qm.y * C.y;
    const T rb = gm.x * B.x + gm.y * B.y + qm.x * D.x + qm.y * D.y;
    part[0] += wy * wz * ra;
    part[1] += dwy * wz * rb;
    part[2] += wy * dwz * rb;
}

// One warp per sorted point k:
//   grad_k = Re[conj(g_k) (grad w_k . U + grad w^o_k . u_f)]
//          + Re[q_k conj(grad w_k . V + grad w^s_k . v_f)]
//          + sum over row k of Re[D w_n],  w_n = conj(g_k) ph_i q_n + q_k conj(ph_i g_n)
// with U, u_f the forward grid potentials of q, V, v_f the adjoint ones of g
// and D = d d_i(k, n) / d r_k from the correction list.  The row constants
// q_k, g_k are folded in per lane, so only three real sums per point are
// reduced over the warp.  Grid sums accumulate in T; the list in FP64
// (DF = false) or in double-float on the FP32 pipes (DF = true, T = float).
template <typename T, int P, bool DF>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 1) grad_kernel(GradArgs a, const cplx<T>* __restrict__ U,
                                                   const cplx<T>* __restrict__ V, const cplx<T>* __restrict__ uf,
                                                   const cplx<T>* __restrict__ vf, const cplx<T>* __restrict__ qs,
                                                   const cplx<T>* __restrict__ gs, double* grad) {
    const int lane = threadIdx.x & 31;
    const long long m = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (m >= a.N) return;
    constexpr int NP = P + 1;
    const cplx<T> qm = qs[m], gm = gs[m];
    T part[3] = {T(0), T(0), T(0)};
    if (lane < NP * NP) {
        const int jy = lane % NP, jz = lane / NP;
        int s[3];
        unpack3(a.ns[m], s[0], s[1], s[2]);
        T t[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) t[d] = sizeof(T) == 8 ? (T)a.ntd[3 * m + d] : (T)a.nt[3 * m + d];
        const long long row = ((long long)(s[2] + jz) * a.n[1] + (s[1] + jy)) * a.n[0] + s[0];
        grad_stencil<T, P>(t, a.h, jy, jz, U + row, V + row, gm, qm, part);
    }
    if (a.has_far) {
        // observer grid for u_f, source grid for v_f
        const int np = a.pf + 1;
        for (int side = 0; side < 2; ++side) {
            int f[3];
            unpack3(side == 0 ? a.fo[m] : a.fs[m], f[0], f[1], f[2]);
            const int toff = side == 0 ? 3 : 0;
            T t[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) t[d] = sizeof(T) == 8 ? (T)a.ftd[6 * m + toff + d] : (T)a.ft[6 * m + toff + d];
            const cplx<T>* gridp = side == 0 ? uf : vf;
            for (int l = lane; l < np * np; l += 32) {
                const int jy = l % np, jz = l / np;
                const cplx<T>* rowp = gridp + ((f[2] + jz) * a.nf[1] + (f[1] + jy)) * a.nf[0] + f[0];
                const cplx<T>* rU = side == 0 ? rowp : nullptr;
                const cplx<T>* rV = side == 0 ? nullptr : rowp;
                if (a.pf == P) grad_stencil<T, P>(t, a.df, jy, jz, rU, rV, gm, qm, part);
                else grad_stencil_rt<T>(a.pf, t, a.df, jy, jz, rU, rV, gm, qm, part);
            }
        }
    }
    // correction list (compact rows: the double-float entries [r0, rb), then
    // the complex64 ones with FP32 derivative heads, summed into the low words)
    const long long r0 = a.row_ptr[m], r1 = a.row_ptr[m + 1];
    const long long rb = DF && a.nbig ? r0 + a.nbig[m] : r1;
    float hh[3] = {0.f, 0.f, 0.f}, ll[3] = {0.f, 0.f, 0.f};  // double-float sums (DF)
    double acc[3] = {0.0, 0.0, 0.0};                         // FP64 sums
    if constexpr (DF) {
        for (long long q = rb + lane; q < r1; q += 32) {
            const uint32_t c = __ldcs(a.col + q);
            const int n = (int)(c & PIM_COL_MASK), ii = (int)(c >> PIM_COL_BITS);
            const cplx<T> xq = qs[n], xg = gs[n];
            float2 D[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) D[d] = __ldcs(a.dvalf + 3 * q + d);
            float ax = (float)xq.x, ay = (float)xq.y, bx = (float)xg.x, by = (float)xg.y;
            if (ii != a.self_img) {
                const float4 ph = a.phasedf[ii];
                const float px = ph.x + ph.y, py = ph.z + ph.w;
                const float tx = px * ax - py * ay, ty = px * ay + py * ax;
                const float ux = px * bx - py * by, uy = px * by + py * bx;
                ax = tx; ay = ty; bx = ux; by = uy;
            }
            const float gx = (float)gm.x, gy = (float)gm.y, qx = (float)qm.x, qy = (float)qm.y;
            const float wr = gx * ax + gy * ay + qx * bx + qy * by;
            const float wi = gx * ay - gy * ax + qy * bx - qx * by;
#pragma unroll
            for (int d = 0; d < 3; ++d) ll[d] += D[d].x * wr - D[d].y * wi;
        }
    }
    for (long long q = r0 + lane; q < rb; q += 32) {
        const uint32_t c = __ldcs(a.col + q);
        const int n = (int)(c & PIM_COL_MASK), ii = (int)(c >> PIM_COL_BITS);
        const cplx<T> xq = qs[n], xg = gs[n];
        if constexpr (DF) {
            float4 D[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) D[d] = __ldcs(a.dvaldf + 3 * q + d);
            float ax = (float)xq.x, ay = (float)xq.y, bx = (float)xg.x, by = (float)xg.y;
            if (ii != a.self_img) {
                const float4 ph = a.phasedf[ii];
                const float px = ph.x + ph.y, py = ph.z + ph.w;
                const float tx = px * ax - py * ay, ty = px * ay + py * ax;
                const float ux = px * bx - py * by, uy = px * by + py * bx;
                ax = tx; ay = ty; bx = ux; by = uy;
            }
            const float gx = (float)gm.x, gy = (float)gm.y, qx = (float)qm.x, qy = (float)qm.y;
            const float wr = gx * ax + gy * ay + qx * bx + qy * by;
            const float wi = gx * ay - gy * ax + qy * bx - qx * by;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                // Re(D w) = D.re w.re - D.im w.im with exact leading products
                const float p1 = D[d].x * wr, e1 = fmaf(D[d].x, wr, -p1);
                const float p2 = D[d].z * wi, e2 = fmaf(D[d].z, wi, -p2);
                two_sum_acc(hh[d], ll[d], p1);
                two_sum_acc(hh[d], ll[d], -p2);
                ll[d] += (e1 - e2) + (D[d].y * wr - D[d].w * wi);
            }
        } else {
            const double2 ph = a.phase[ii];
            const double2 pq = cmul(ph, make_double2((double)xq.x, (double)xq.y));  // ph q_n
            const double2 pg = cmul(ph, make_double2((double)xg.x, (double)xg.y));  // ph g_n
            const double2 gmd = make_double2((double)gm.x, (double)gm.y), qmd = make_double2((double)qm.x, (double)qm.y);
            const double2 w = cadd(cmul(cconj(gmd), pq), cmul(qmd, cconj(pg)));
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double2 Dd = a.dval[3 * q + d];
                acc[d] += Dd.x * w.x - Dd.y * w.y;
            }
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) part[d] += __shfl_xor_sync(0xffffffffu, part[d], o);
        if constexpr (DF) {
            df_warp_sum(hh[d], ll[d]);
        } else {
            for (int o = 16; o > 0; o >>= 1) acc[d] += __shfl_xor_sync(0xffffffffu, acc[d], o);
        }
    }
    if (lane == 0) {
        for (int d = 0; d < 3; ++d) {
            double v;
            if constexpr (DF) {
                // part + hh + ll in FP32 (TwoSum), one conversion
                float s, e;
                two_sum((float)part[d], hh[d], s, e);
                v = (double)s + (double)(e + ll[d]);
            } else {
                v = (double)part[d] + acc[d];
            }
            const long long o = 3LL * a.perm[m] + d;
            grad[o] = a.first ? v : grad[o] + v;
        }
    }
}

// u[perm[m]] = us[m] - mean  (the adjoint of the neutral static case)
template <typename T>
__global__ void unpermute_kernel(const cplx<T>* us, const int* perm, long long N, int nrhs, int r, const double* mean,
                                 int real_out, void* out) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const double re = (double)us[m].x - mean[0], im = (double)us[m].y - mean[1];
        const long long o = (long long)perm[m] * nrhs + r;
        if (real_out) ((T*)out)[o] = (T)re;
        else ((cplx<T>*)out)[o] = mk<T>((T)re, (T)im);
    }
}

// ------------------------------- multi-RHS correction ----------------------
// u[perm[m]][r] += sum_row exp(-j k0.(i o L)) d q_n[r] (conj(d) for the
// adjoint) for every right-hand side r: one warp per sorted row, lanes over
// right-hand sides; each entry's column and value are loaded once (broadcast)
// and used for all right-hand sides, the sources q_n[0..R) are one coalesced
// row.  Accumulation as in the single-RHS kernel (FP64, double-float or FP32).
struct CorrMultiArgs {
    long long N;
    int nrhs, adj, self_img, real_out;
    const int* perm;
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

// a value of lane `src`, for the broadcast of list values inside a warp
__device__ __forceinline__ float2 shfl_value(float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ __forceinline__ float4 shfl_value(float4 v, int src) {
    return make_float4(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src),
                       __shfl_sync(0xffffffffu, v.z, src), __shfl_sync(0xffffffffu, v.w, src));
}
__device__ __forceinline__ double2 shfl_value(double2 v, int src) {
    return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

template <typename T, int CM, int RPL>
__global__ void __launch_bounds__(256) corr_multi_kernel(CorrMultiArgs a, const cplx<T>* __restrict__ qsall, void* out) {
    const int lane = threadIdx.x & 31;
    const long long m = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (m >= a.N) return;
    const int R = a.nrhs;
    double2 acc[RPL];
    float rh[RPL], rl[RPL], ih[RPL], il[RPL];
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        acc[k] = make_double2(0.0, 0.0);
        rh[k] = rl[k] = ih[k] = il[k] = 0.f;
    }
    const double cs = a.adj ? -1.0 : 1.0;
    const float fs = (float)cs;
    const long long r0 = a.row_ptr[m], r1 = a.row_ptr[m + 1];
    // The row in groups of 32 entries: lane j loads entry j's column and
    // value and applies its image phase, then the warp walks the group's
    // entries with the column and value broadcast by shuffles; the source
    // loads of consecutive entries are independent, so several are in flight.
    auto group = [&](long long s0, long long s1, auto load_v, auto mac) {
        for (long long q0 = s0; q0 < s1; q0 += 32) {
            const long long q = q0 + lane < s1 ? q0 + lane : s1 - 1;
            const int cnt = (int)(s1 - q0 < 32 ? s1 - q0 : 32);
            const uint32_t c = __ldg(a.col + q);
            const int nl = (int)(c & PIM_COL_MASK);
            const auto v = load_v(q, (int)(c >> PIM_COL_BITS));
#pragma unroll 4
            for (int e = 0; e < cnt; ++e) {
                const int n = __shfl_sync(0xffffffffu, nl, e);
                const auto ve = shfl_value(v, e);
                const cplx<T>* xr = qsall + (long long)n * R;
#pragma unroll
                for (int k = 0; k < RPL; ++k) {
                    const int r = lane + 32 * k;
                    if (r < R) mac(k, ve, xr[r]);
                }
            }
        }
    };
    // double-float entries: all of them, or a compact row's leading ones
    const long long rb = CM == PIM_CORR_COMPACT ? r0 + a.nbig[m] : r1;
    if (corr_df(CM)) {
        group(r0, rb,
              [&](long long q, int ii) {
                  const float4 d = CM == PIM_CORR_COMPACT ? compact_value(__ldg(a.valf + q), __ldg(a.valt + q))
                                                          : __ldg(a.valdf + q);
                  float4 v = make_float4(d.x, d.y, fs * d.z, fs * d.w);
                  if (ii != a.self_img) v = df_cmul(a.phasedf[ii], v);
                  return v;
              },
              [&](int k, const float4& v, const cplx<T>& xv) {
                  df_cmac(rh[k], rl[k], ih[k], il[k], v, (float)xv.x, (float)xv.y);
              });
    }
    // complex64 entries: all of them, or a compact row's trailing ones (their
    // sums go to the low words)
    if (CM == PIM_CORR_FP32 || CM == PIM_CORR_COMPACT) {
        group(CM == PIM_CORR_COMPACT ? rb : r0, r1,
              [&](long long q, int ii) {
                  const float2 d = __ldg(a.valf + q);
                  float2 dd = make_float2(d.x, fs * d.y);
                  if (ii != a.self_img) {
                      const double2 ph = a.phase[ii];
                      dd = make_float2((float)ph.x * dd.x - (float)ph.y * dd.y, (float)ph.x * dd.y + (float)ph.y * dd.x);
                  }
                  return dd;
              },
              [&](int k, const float2& dd, const cplx<T>& xv) {
                  const float tr = dd.x * (float)xv.x - dd.y * (float)xv.y;
                  const float ti = dd.x * (float)xv.y + dd.y * (float)xv.x;
                  if (CM == PIM_CORR_COMPACT) {
                      rl[k] += tr;
                      il[k] += ti;
                  } else {
                      rh[k] += tr;
                      ih[k] += ti;
                  }
              });
    }
    if (CM == PIM_CORR_FP64) {
        group(r0, r1,
              [&](long long q, int ii) {
                  double2 d = __ldg(a.val + q);
                  d.y *= cs;
                  if (ii != a.self_img) d = cmul(a.phase[ii], d);
                  return d;
              },
              [&](int k, const double2& d, const cplx<T>& xv) {
                  acc[k].x += d.x * (double)xv.x - d.y * (double)xv.y;
                  acc[k].y += d.x * (double)xv.y + d.y * (double)xv.x;
              });
    }
    const long long o = (long long)a.perm[m] * R;
#pragma unroll
    for (int k = 0; k < RPL; ++k) {
        const int r = lane + 32 * k;
        if (r >= R) break;
        const double re = acc[k].x + (double)rh[k] + (double)rl[k];
        const double im = acc[k].y + (double)ih[k] + (double)il[k];
        if (a.real_out) {
            T* u = (T*)out + o + r;
            *u = (T)((double)*u + re);
        } else {
            cplx<T>* u = (cplx<T>*)out + o + r;
            cplx<T> v = *u;
            v.x = (T)((double)v.x + re);
            v.y = (T)((double)v.y + im);
            *u = v;
        }
    }
}

// qsall[m][r] = q[perm[m]][r] - mean[r] for all right-hand sides
template <typename T, bool REAL>
__global__ void permute_all_kernel(const void* q, const int* perm, long long N, int nrhs, const double* means,
                                   cplx<T>* qsall) {
    const long long tot = N * nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long m = e / nrhs;
        const int r = (int)(e % nrhs);
        const double2 v = load_val<T, REAL>(q, (long long)perm[m] * nrhs + r);
        const double mr = means ? means[2 * r] : 0.0, mi = means ? means[2 * r + 1] : 0.0;
        qsall[e] = mk<T>((T)(v.x - mr), (T)(v.y - mi));
    }
}

__global__ void copy_mean_kernel(const double* src, double* dst) {
    dst[0] = src[0];
    dst[1] = src[1];
}

// ------------------------------- driver ------------------------------------
template <typename T>
pim_status mean_of(pim_plan P, const void* q, bool sorted_complex, long long N, int nrhs, int r, bool check,
                   cudaStream_t s) {
    double* partial = P->dsum + 4;
    if (sorted_complex) sum_partials_kernel<T, false><<<RED_BLOCKS, RED_NT, 0, s>>>(q, N, 1, 0, partial);
    else if (P->real_data) sum_partials_kernel<T, true><<<RED_BLOCKS, RED_NT, 0, s>>>(q, N, nrhs, r, partial);
    else sum_partials_kernel<T, false><<<RED_BLOCKS, RED_NT, 0, s>>>(q, N, nrhs, r, partial);
    sum_final_kernel<<<1, RED_NT, 0, s>>>(partial, RED_BLOCKS, N, P->neutral_tol, check ? 1 : 0, P->dsum,
                                          P->dstatus);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <typename T, int PP>
pim_status run_typed(pim_plan P, const void* q, void* u, int nrhs, bool adj, cudaStream_t s) {
    const PointsData& d = P->pts;
    const long long N = d.N;
    cplx<T>* qs = (cplx<T>*)P->qs;
    cplx<T>* gA = (cplx<T>*)P->gA;
    pim_status st;
    // several right-hand sides: the per-RHS gathers skip the correction and one
    // multi-RHS kernel adds it for all of them (the list is streamed once)
    const bool multi = nrhs > 1 && nrhs <= 128 && !P->no_multi && !(P->npsp && adj) && N > 0;
    if (multi) {
        const size_t need = (size_t)N * nrhs * sizeof(cplx<T>);
        if (P->qsall_bytes < need) {
            pim_free(P, P->qsall, P->qsall_bytes);
            P->qsall = nullptr;
            P->qsall_bytes = 0;
            if ((st = pim_alloc(P, &P->qsall, need)) != PIM_OK) return st;
            P->qsall_bytes = need;
        }
        if (!P->dmeans && (st = pim_alloc(P, (void**)&P->dmeans, 2 * 128 * sizeof(double))) != PIM_OK) return st;
    }
    // the right-hand sides of a multi-RHS apply go round-robin to lanes with
    // their own scratch and streams, so that several run at once
    // (not for the neutral static case, whose per-RHS means share one scratch)
    const int K = multi && !P->npsp ? std::min(nrhs, (int)pim_plan_s::RHS_LANES) : 1;
    // plans with the position gradient keep the grid potentials of their last
    // single-RHS forward (near in gA, far in fU) and adjoint (gD, fV) applies
    const bool keep = P->with_gradient && nrhs == 1 && !multi && !P->keep_off && P->gD;
    const int kept = P->pot_valid;
    P->pot_valid = 0;  // until this apply has been issued in full
    const int prof_slot0 = P->prof_next;  // ring slot of this call's first right-hand side
    if (K > 1) {
        if ((st = lanes_prepare(P, K)) != PIM_OK) return st;
        PIM_CK(cudaEventRecord(P->lane_fork, s));
        for (int k = 1; k < K; ++k) PIM_CK(cudaStreamWaitEvent(P->lane[k].sm, P->lane_fork, 0));
    }
    const pim_plan_s::Lane own{P->qs, P->gA, P->gB, P->gC, P->pts.mom, P->fpart, P->fA, P->fB, P->fC, P->ufp,
                               s, P->s_far, P->ev_fork, P->ev_join, nullptr};
    auto use_lane = [&](const pim_plan_s::Lane& l) {
        P->qs = l.qs; P->gA = l.gA; P->gB = l.gB; P->gC = l.gC; P->pts.mom = l.mom; P->fpart = l.fpart;
        P->fA = l.fA; P->fB = l.fB; P->fC = l.fC; P->ufp = l.ufp; P->s_far = l.sf; P->ev_fork = l.fork;
        P->ev_join = l.join;
    };
    // the plan's own scratch is back in place on every way out
    struct Restore {
        decltype(use_lane)& f;
        const pim_plan_s::Lane& l;
        ~Restore() { f(l); }
    } restore{use_lane, own};
    for (int r = 0; r < nrhs; ++r) {
        const int lk = r % K;
        use_lane(lk == 0 ? own : P->lane[lk]);
        const cudaStream_t sr = lk == 0 ? s : P->lane[lk].sm;
        qs = (cplx<T>*)P->qs;
        gA = (cplx<T>*)P->gA;
        cplx<T>* gN = keep && adj ? (cplx<T>*)P->gD : gA;  // the near grid of this apply
        prof_mark(P, PIM_STAGE_APPLY, 0, sr);
        prof_mark(P, PIM_STAGE_PERMUTE, 0, sr);
        // 1. sorted, regularised sources (Eq. neutral)
        const double* mean = nullptr;
        if (P->npsp && !adj) {
            if ((st = mean_of<T>(P, q, false, N, nrhs, r, true, sr)) != PIM_OK) return st;
            mean = P->dsum;
            if (multi) copy_mean_kernel<<<1, 1, 0, sr>>>(P->dsum, P->dmeans + 2 * r);
        }
        if (P->real_data) permute_kernel<T, true><<<1024, 256, 0, sr>>>(q, d.perm, N, nrhs, r, mean, qs);
        else permute_kernel<T, false><<<1024, 256, 0, sr>>>(q, d.perm, N, nrhs, r, mean, qs);
        PIM_CK(cudaGetLastError());
        P->launches += 1 + (mean ? 2 : 0);
        prof_mark(P, PIM_STAGE_PERMUTE, 1, sr);
        // 2. far zone on the second stream
        if (P->has_far) {
            PIM_CK(cudaEventRecord(P->ev_fork, sr));
            PIM_CK(cudaStreamWaitEvent(P->s_far, P->ev_fork, 0));
            prof_mark(P, PIM_STAGE_FAR, 0, P->s_far);
            const int G = P->nf[0] * P->nf[1] * P->nf[2];
            if ((st = far_spread_grid<T>(P, N, adj ? d.fo : d.fs, adj ? 3 : 0, qs, P->fA, P->s_far)) != PIM_OK)
                return st;
            if ((st = fft3_conv<double>(P, P->fg, P->fA, P->fB, P->fC, P->fspec, adj, P->s_far)) != PIM_OK) return st;
            if (sizeof(T) == 4) {
                far_convert_kernel<T><<<(G + 255) / 256, 256, 0, P->s_far>>>(P->fA, (cplx<T>*)P->fB, G);
                PIM_CK(cudaGetLastError());
            }
            if (keep) {
                far_convert_kernel<T><<<(G + 255) / 256, 256, 0, P->s_far>>>(P->fA, (cplx<T>*)(adj ? P->fV : P->fU), G);
                PIM_CK(cudaGetLastError());
                P->launches += 1;
            }
            // far gather of every point (Eq. interpolation), while the near
            // path and its gather run on the main stream
            if (N > 0) {
                GatherArgs fg{};
                for (int i = 0; i < 3; ++i) fg.nf[i] = P->nf[i];
                fg.pf = P->pf;
                fg.N = N;
                fg.fst = adj ? d.fs : d.fo;
                fg.ft = d.ft;
                fg.ftd = d.ftd;
                fg.toff = adj ? 0 : 3;
                fg.perm = d.perm;
                const cplx<T>* ufar = sizeof(T) == 4 ? (const cplx<T>*)P->fB : (const cplx<T>*)P->fA;
                if ((st = launch_far_interp<T>(P->pf, N, P->s_far, fg, ufar, (cplx<T>*)P->ufp)) != PIM_OK) return st;
            }
            P->launches += 5 + (sizeof(T) == 4 ? 1 : 0) + (N > 0 ? 1 : 0);
            prof_mark(P, PIM_STAGE_FAR, 1, P->s_far);
            PIM_CK(cudaEventRecord(P->ev_join, P->s_far));
        }
        // list-free boxes, one right-hand side: their exact part on its own
        // stream, while the spread, FFT and gather run
        const bool lf_async = P->pts.nlf > 0 && P->ulf && nrhs == 1 && N > 0;
        // with the tensor-core form the grid part runs on this stream after the
        // gather: it moves the local grids through HBM, and beside the gather
        // and FFT it would slow them by more than it takes alone
        const bool grid_main = lf_async && P->pts.ntc > 0;
        if (lf_async) {
            PIM_CK(cudaEventRecord(P->ev_lf_fork, sr));
            PIM_CK(cudaStreamWaitEvent(P->s_lf, P->ev_lf_fork, 0));
            if ((st = lf_exact_async(P, qs, adj, P->s_lf)) != PIM_OK) return st;
            if (grid_main) PIM_CK(cudaEventRecord(P->ev_lf_join, P->s_lf));
        }
        // 3. near spread (two phases), 4. FFT convolution
        prof_mark(P, PIM_STAGE_SPREAD, 0, sr);
        if ((st = spread_two_phase<T, PP>(P, qs, gN, sr)) != PIM_OK) return st;
        prof_mark(P, PIM_STAGE_SPREAD, 1, sr);
        // the list-free boxes' grid part needs the box moments of the spread
        if (lf_async && !grid_main) {
            PIM_CK(cudaEventRecord(P->ev_lf_mom, sr));
            PIM_CK(cudaStreamWaitEvent(P->s_lf, P->ev_lf_mom, 0));
            if ((st = lf_grid_async(P, qs, adj, P->s_lf)) != PIM_OK) return st;
            PIM_CK(cudaEventRecord(P->ev_lf_join, P->s_lf));
        }
        prof_mark(P, PIM_STAGE_FFT, 0, sr);
        if ((st = fft3_conv<T>(P, P->ng, gN, (cplx<T>*)P->gB, (cplx<T>*)P->gC, (const cplx<T>*)P->spec, adj, sr)) != PIM_OK)
            return st;
        prof_mark(P, PIM_STAGE_FFT, 1, sr);
        P->launches += (d.nd > 0 ? 2 : 1) + 5;
        // 5. gather + correction, then the far part once both streams joined
        GatherArgs ga{};
        for (int i = 0; i < 3; ++i) { ga.n[i] = P->n[i]; ga.nf[i] = P->nf[i]; }
        ga.pf = P->pf;
        ga.N = N;
        ga.nrhs = nrhs;
        ga.r = r;
        ga.cmode = multi ? -1 : (sizeof(T) == 8 ? PIM_CORR_FP64 : P->corr_mode);
        ga.adj = adj ? 1 : 0;
        ga.has_far = P->has_far ? 1 : 0;
        ga.real_out = P->real_data ? 1 : 0;
        const bool post_mean = P->npsp && adj;
        ga.sorted_out = post_mean ? 1 : 0;
        ga.self_img = -1;
        for (int i = 0; i < P->nimg; ++i)
            if (P->img[i][0] == 0 && P->img[i][1] == 0 && P->img[i][2] == 0) ga.self_img = i;
        ga.perm = d.perm;
        ga.ns = d.ns;
        ga.nt = d.nt;
        ga.ntd = d.ntd;
        ga.fst = adj ? d.fs : d.fo;
        ga.ft = d.ft;
        ga.ftd = d.ftd;
        ga.toff = adj ? 0 : 3;
        ga.row_ptr = d.row_ptr;
        ga.col = d.col;
        ga.val = d.val;
        ga.valdf = d.valdf;
        ga.valf = d.valf;
        ga.valt = d.valt;
        ga.nbig = d.nbig;
        ga.phase = adj ? P->dphase_adj : P->dphase;
        ga.phasedf = adj ? P->dphasedf_adj : P->dphasedf;
        void* dst = post_mean ? P->us : u;
        const long long threads = N * 32;
        prof_mark(P, PIM_STAGE_GATHER, 0, sr);
        if (N > 0) {
            const unsigned nb = (unsigned)((threads + 255) / 256);
            if (P->tune_ev[0]) PIM_CK(cudaEventRecord(P->tune_ev[0], sr));
            if ((st = launch_gather<T, PP>(ga.cmode, P->gather_variant, nb, sr, ga, gN, qs, dst)) != PIM_OK)
                return st;
            if (P->tune_ev[1]) PIM_CK(cudaEventRecord(P->tune_ev[1], sr));
        }
        PIM_CK(cudaGetLastError());
        prof_mark(P, PIM_STAGE_GATHER, 1, sr);
        P->launches += N > 0 ? 1 : 0;
        // list-free boxes: exact sum minus grid part, added to the gathered output
        if (lf_async) {
            PIM_CK(cudaStreamWaitEvent(sr, P->ev_lf_join, 0));
            if (grid_main && (st = lf_grid_async(P, qs, adj, sr)) != PIM_OK) return st;
            if ((st = lf_add(P, dst, post_mean, sr)) != PIM_OK) return st;
        } else if (N > 0 && (st = lf_apply(P, qs, dst, nrhs, r, adj, post_mean, sr, lk)) != PIM_OK) {
            return st;
        }
        if (P->has_far) {
            PIM_CK(cudaStreamWaitEvent(sr, P->ev_join, 0));
            if (N > 0) {
                far_add_kernel<T><<<(unsigned)std::min<long long>((N + 255) / 256, 152 * 8), 256, 0, sr>>>(
                    ga, (const cplx<T>*)P->ufp, dst);
                PIM_CK(cudaGetLastError());
                P->launches += 1;
            }
        }
        if (post_mean) {
            if ((st = mean_of<T>(P, P->us, true, N, 1, 0, false, sr)) != PIM_OK) return st;
            unpermute_kernel<T><<<1024, 256, 0, sr>>>((const cplx<T>*)P->us, d.perm, N, nrhs, r, P->dsum,
                                                     P->real_data ? 1 : 0, u);
            PIM_CK(cudaGetLastError());
            P->launches += 3;
        }
        prof_mark(P, PIM_STAGE_APPLY, 1, sr);
        if (P->prof_on && P->prof_next < pim_plan_s::PROF_RING) P->prof_next++;
    }
    use_lane(own);
    qs = (cplx<T>*)P->qs;
    gA = (cplx<T>*)P->gA;
    for (int k = 1; k < K; ++k) {
        PIM_CK(cudaEventRecord(P->lane[k].done, P->lane[k].sm));
        PIM_CK(cudaStreamWaitEvent(s, P->lane[k].done, 0));
    }
    if (multi) {
        cplx<T>* qsall = (cplx<T>*)P->qsall;
        const double* means = (P->npsp && !adj) ? P->dmeans : nullptr;
        if (P->real_data) permute_all_kernel<T, true><<<1024, 256, 0, s>>>(q, d.perm, N, nrhs, means, qsall);
        else permute_all_kernel<T, false><<<1024, 256, 0, s>>>(q, d.perm, N, nrhs, means, qsall);
        CorrMultiArgs ca{};
        ca.N = N;
        ca.nrhs = nrhs;
        ca.adj = adj ? 1 : 0;
        ca.self_img = -1;
        for (int i = 0; i < P->nimg; ++i)
            if (P->img[i][0] == 0 && P->img[i][1] == 0 && P->img[i][2] == 0) ca.self_img = i;
        ca.real_out = P->real_data ? 1 : 0;
        ca.perm = d.perm;
        ca.row_ptr = d.row_ptr;
        ca.col = d.col;
        ca.val = d.val;
        ca.valdf = d.valdf;
        ca.valf = d.valf;
        ca.valt = d.valt;
        ca.nbig = d.nbig;
        ca.phase = adj ? P->dphase_adj : P->dphase;
        ca.phasedf = adj ? P->dphasedf_adj : P->dphasedf;
        const int cm = sizeof(T) == 8 ? PIM_CORR_FP64 : P->corr_mode;
        const unsigned nb = (unsigned)((N * 32 + 255) / 256);
        // timed in the ring slot of the last right-hand side, if this call recorded any
        const bool prof_corr = P->prof_on && P->prof_next > prof_slot0;
        if (prof_corr) --P->prof_next;
        prof_mark(P, PIM_STAGE_CORR_MULTI, 0, s);
#define PIM_CM_LAUNCH(CMV)                                                                                   \
    do {                                                                                                     \
        if (nrhs <= 32) corr_multi_kernel<T, CMV, 1><<<nb, 256, 0, s>>>(ca, qsall, u);                      \
        else if (nrhs <= 64) corr_multi_kernel<T, CMV, 2><<<nb, 256, 0, s>>>(ca, qsall, u);                 \
        else corr_multi_kernel<T, CMV, 4><<<nb, 256, 0, s>>>(ca, qsall, u);                                 \
    } while (0)
        if (cm == PIM_CORR_COMPACT) PIM_CM_LAUNCH(PIM_CORR_COMPACT);
        else if (cm == PIM_CORR_DOUBLE_FLOAT) PIM_CM_LAUNCH(PIM_CORR_DOUBLE_FLOAT);
        else if (cm == PIM_CORR_FP32) PIM_CM_LAUNCH(PIM_CORR_FP32);
        else PIM_CM_LAUNCH(PIM_CORR_FP64);
#undef PIM_CM_LAUNCH
        PIM_CK(cudaGetLastError());
        prof_mark(P, PIM_STAGE_CORR_MULTI, 1, s);
        if (prof_corr) ++P->prof_next;
        P->launches += 2;
    }
    if (keep) P->pot_valid = kept | (adj ? 2 : 1);
    return PIM_OK;
}

template <typename T>
pim_status run_p(pim_plan P, const void* q, void* u, int nrhs, bool adj, cudaStream_t s) {
    switch (P->p) {
        case 2: return run_typed<T, 2>(P, q, u, nrhs, adj, s);
        case 3: return run_typed<T, 3>(P, q, u, nrhs, adj, s);
        case 4: return run_typed<T, 4>(P, q, u, nrhs, adj, s);
        default: pim_set_error("GPU path supports p = 2, 3, 4"); return PIM_ERR_UNSUPPORTED;
    }
}

template <typename T, int PP>
pim_status grad_typed(pim_plan P, const void* q, const void* g, double* grad, int nrhs, cudaStream_t s,
                      bool reuse) {
    const PointsData& d = P->pts;
    const long long N = d.N;
    cplx<T>* qs = (cplx<T>*)P->qs;
    cplx<T>* gs = (cplx<T>*)P->gsrt;
    cplx<T>* gA = (cplx<T>*)P->gA;
    cplx<T>* gD = (cplx<T>*)P->gD;
    const int G = P->has_far ? P->nf[0] * P->nf[1] * P->nf[2] : 0;
    pim_status st;
    for (int r = 0; r < nrhs; ++r) {
        const double* mean = nullptr;
        if (P->npsp) {
            if ((st = mean_of<T>(P, q, false, N, nrhs, r, true, s)) != PIM_OK) return st;
            mean = P->dsum;
        }
        if (P->real_data) {
            permute_kernel<T, true><<<1024, 256, 0, s>>>(q, d.perm, N, nrhs, r, mean, qs);
            permute_kernel<T, true><<<1024, 256, 0, s>>>(g, d.perm, N, nrhs, r, nullptr, gs);
        } else {
            permute_kernel<T, false><<<1024, 256, 0, s>>>(q, d.perm, N, nrhs, r, mean, qs);
            permute_kernel<T, false><<<1024, 256, 0, s>>>(g, d.perm, N, nrhs, r, nullptr, gs);
        }
        PIM_CK(cudaGetLastError());
        // far grid potentials: u_f from the source-grid projection of q, v_f
        // (adjoint) from the observer-grid projection of g, on the far
        // stream while the near grids are built (reuse: those the last
        // forward and adjoint applies left in fU, fV, gA and gD)
        if (P->has_far && !reuse) {
            PIM_CK(cudaEventRecord(P->ev_fork, s));
            PIM_CK(cudaStreamWaitEvent(P->s_far, P->ev_fork, 0));
            for (int side = 0; side < 2; ++side) {
                double2* fq = side == 0 ? P->fA : P->fD;
                if ((st = far_spread_grid<T>(P, N, side == 0 ? d.fs : d.fo, side == 0 ? 0 : 3, side == 0 ? qs : gs, fq,
                                             P->s_far)) != PIM_OK)
                    return st;
                if ((st = fft3_conv<double>(P, P->fg, fq, P->fB, P->fC, P->fspec, side == 1, P->s_far)) != PIM_OK) return st;
                far_convert_kernel<T><<<(G + 255) / 256, 256, 0, P->s_far>>>(fq, (cplx<T>*)(side == 0 ? P->fU : P->fV), G);
                PIM_CK(cudaGetLastError());
            }
            PIM_CK(cudaEventRecord(P->ev_join, P->s_far));
        }
        // near grid potentials: U = K * Q(q), V = K^H * Q(g)
        if (!reuse) {
            P->pot_valid = 0;  // gA and gD no longer hold the applies' potentials
            if ((st = spread_two_phase<T, PP>(P, qs, gA, s)) != PIM_OK) return st;
            if ((st = fft3_conv<T>(P, P->ng, gA, (cplx<T>*)P->gB, (cplx<T>*)P->gC, (const cplx<T>*)P->spec, false,
                                   s)) != PIM_OK)
                return st;
            if ((st = spread_two_phase<T, PP>(P, gs, gD, s)) != PIM_OK) return st;
            if ((st = fft3_conv<T>(P, P->ng, gD, (cplx<T>*)P->gB, (cplx<T>*)P->gC, (const cplx<T>*)P->spec, true,
                                   s)) != PIM_OK)
                return st;
            if (P->has_far) PIM_CK(cudaStreamWaitEvent(s, P->ev_join, 0));
        }
        GradArgs ga{};
        for (int i = 0; i < 3; ++i) {
            ga.n[i] = P->n[i];
            ga.nf[i] = P->nf[i];
            ga.h[i] = P->h[i];
            ga.df[i] = P->df[i];
        }
        ga.pf = P->pf;
        ga.N = N;
        ga.has_far = P->has_far ? 1 : 0;
        ga.self_img = -1;
        ga.first = r == 0 ? 1 : 0;
        ga.perm = d.perm;
        ga.ns = d.ns;
        ga.nt = d.nt;
        ga.ntd = d.ntd;
        ga.fs = d.fs;
        ga.fo = d.fo;
        ga.ft = d.ft;
        ga.ftd = d.ftd;
        ga.row_ptr = d.row_ptr;
        ga.col = d.col;
        ga.dval = d.dval;
        ga.dvaldf = reinterpret_cast<const float4*>(d.dval);
        ga.dvalf = d.dvalf;
        ga.nbig = P->corr_mode == PIM_CORR_COMPACT ? d.nbig : nullptr;
        ga.phase = P->dphase;
        ga.phasedf = P->dphasedf;
        for (int i = 0; i < P->nimg; ++i)
            if (P->img[i][0] == 0 && P->img[i][1] == 0 && P->img[i][2] == 0) ga.self_img = i;
        const unsigned nbk = (unsigned)((N * 32 + 255) / 256);
        if (N > 0) {
            if constexpr (sizeof(T) == 4) {
                if (corr_df(P->corr_mode))
                    grad_kernel<T, PP, true><<<nbk, 256, 0, s>>>(ga, gA, gD, (const cplx<T>*)P->fU,
                                                                 (const cplx<T>*)P->fV, qs, gs, grad);
                else
                    grad_kernel<T, PP, false><<<nbk, 256, 0, s>>>(ga, gA, gD, (const cplx<T>*)P->fU,
                                                                  (const cplx<T>*)P->fV, qs, gs, grad);
            } else {
                grad_kernel<T, PP, false><<<nbk, 256, 0, s>>>(ga, gA, gD, (const cplx<T>*)P->fU,
                                                              (const cplx<T>*)P->fV, qs, gs, grad);
            }
        }
        PIM_CK(cudaGetLastError());
    }
    return PIM_OK;
}

template <typename T>
pim_status grad_p(pim_plan P, const void* q, const void* g, double* grad, int nrhs, cudaStream_t s, bool reuse) {
    switch (P->p) {
        case 2: return grad_typed<T, 2>(P, q, g, grad, nrhs, s, reuse);
        case 3: return grad_typed<T, 3>(P, q, g, grad, nrhs, s, reuse);
        case 4: return grad_typed<T, 4>(P, q, g, grad, nrhs, s, reuse);
        default: return PIM_ERR_UNSUPPORTED;
    }
}

template <typename T, int PP>
pim_status debug_spread_typed(pim_plan P, void* out, cudaStream_t s) {
    return spread_two_phase<T, PP>(P, (const cplx<T>*)P->qs, (cplx<T>*)out, s);
}

template <typename T>
pim_status debug_spread_p(pim_plan P, void* out, cudaStream_t s) {
    switch (P->p) {
        case 2: return debug_spread_typed<T, 2>(P, out, s);
        case 3: return debug_spread_typed<T, 3>(P, out, s);
        case 4: return debug_spread_typed<T, 4>(P, out, s);
        default: return PIM_ERR_UNSUPPORTED;
    }
}

}  // namespace

pim_status grad_run(pim_plan P, const void* q, const void* g, double* grad, int nrhs, cudaStream_t s, bool reuse) {
    if (P->prec == PIM_FP64) return grad_p<double>(P, q, g, grad, nrhs, s, reuse);
    return grad_p<float>(P, q, g, grad, nrhs, s, reuse);
}

pim_status apply_debug_spread(pim_plan P, void* out, cudaStream_t s) {
    if (P->prec == PIM_FP64) return debug_spread_p<double>(P, out, s);
    return debug_spread_p<float>(P, out, s);
}

// Allocates what an apply with these arguments would allocate on first use
// (the multi-RHS source buffer), so that the apply itself can be captured.
// Scratch sizes of one right-hand-side lane (the per-RHS buffers of an apply).
static void lane_sizes(pim_plan P, size_t* sz) {
    const size_t ge = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t N = (size_t)P->pts.N;
    const size_t G = (size_t)P->n[0] * P->n[1] * P->n[2];
    const size_t GB = (size_t)P->n[2] * P->n[1] * P->ng.L[0];
    const size_t GC = (size_t)P->n[2] * P->ng.L[1] * P->ng.L[0];
    const size_t np3 = (size_t)(P->p + 1) * (P->p + 1) * (P->p + 1);
    size_t Gf = 0, fB = 0, fC = 0;
    if (P->has_far) {
        Gf = (size_t)P->nf[0] * P->nf[1] * P->nf[2];
        fB = (size_t)P->nf[2] * P->nf[1] * P->fg.L[0];
        fC = (size_t)P->nf[2] * P->fg.L[1] * P->fg.L[0];
    }
    sz[0] = N * ge;
    sz[1] = G * ge;
    sz[2] = GB * ge;
    sz[3] = GC * ge;
    sz[4] = (size_t)(P->pts.nd > 0 ? P->pts.nd : 1) * np3 * ge;
    sz[5] = (size_t)P->far_chunks * Gf * ge;
    sz[6] = Gf * sizeof(double2);
    sz[7] = fB * sizeof(double2);
    sz[8] = fC * sizeof(double2);
    sz[9] = P->has_far ? N * ge : 0;
}

void lanes_free(pim_plan P) {
    size_t sz[10];
    lane_sizes(P, sz);
    for (int k = 1; k < P->nlanes; ++k) {
        pim_plan_s::Lane& l = P->lane[k];
        void* b[10] = {l.qs, l.gA, l.gB, l.gC, l.mom, l.fpart, l.fA, l.fB, l.fC, l.ufp};
        for (int i = 0; i < 10; ++i) pim_free(P, b[i], sz[i]);
        if (l.sm) cudaStreamDestroy(l.sm);
        if (l.sf) cudaStreamDestroy(l.sf);
        if (l.fork) cudaEventDestroy(l.fork);
        if (l.join) cudaEventDestroy(l.join);
        if (l.done) cudaEventDestroy(l.done);
        l = pim_plan_s::Lane{};
    }
    P->nlanes = 1;
}

pim_status lanes_prepare(pim_plan P, int nl) {
    nl = std::min(nl, (int)pim_plan_s::RHS_LANES);
    if (P->nlanes >= nl) return PIM_OK;
    if (!P->lane_fork && cudaEventCreateWithFlags(&P->lane_fork, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        pim_set_error("event creation failed");
        return PIM_ERR_CUDA;
    }
    size_t sz[10];
    lane_sizes(P, sz);
    for (int k = P->nlanes; k < nl; ++k) {
        pim_plan_s::Lane& l = P->lane[k];
        void** b[10] = {&l.qs, &l.gA, &l.gB, &l.gC, &l.mom, &l.fpart, (void**)&l.fA, (void**)&l.fB, (void**)&l.fC,
                        &l.ufp};
        pim_status st;
        for (int i = 0; i < 10; ++i)
            if (sz[i] && (st = pim_alloc(P, b[i], sz[i])) != PIM_OK) return st;
        if (cudaStreamCreateWithFlags(&l.sm, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithPriority(&l.sf, cudaStreamNonBlocking, far_stream_priority()) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.join, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&l.done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            pim_set_error("stream or event creation failed");
            return PIM_ERR_CUDA;
        }
        P->nlanes = k + 1;
    }
    return PIM_OK;
}

pim_status apply_prepare(pim_plan P, int nrhs, bool adj) {
    const long long N = P->pts.N;
    const bool multi = nrhs > 1 && nrhs <= 128 && !P->no_multi && !(P->npsp && adj) && N > 0;
    if (!multi) return PIM_OK;
    pim_status st;
    if (!P->npsp && (st = lanes_prepare(P, std::min(nrhs, (int)pim_plan_s::RHS_LANES))) != PIM_OK) return st;
    const size_t el = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t need = (size_t)N * nrhs * el;
    if (P->qsall_bytes < need) {
        pim_free(P, P->qsall, P->qsall_bytes);
        P->qsall = nullptr;
        P->qsall_bytes = 0;
        if ((st = pim_alloc(P, &P->qsall, need)) != PIM_OK) return st;
        P->qsall_bytes = need;
    }
    if (!P->dmeans && (st = pim_alloc(P, (void**)&P->dmeans, 2 * 128 * sizeof(double))) != PIM_OK) return st;
    return PIM_OK;
}

// Launch shapes of the gather kernel: (unroll depth of the row loop, minimum
// resident CTAs), the same set for every precision and correction mode.
int gather_variant_count(const pim_plan_s*) { return GATHER_VARIANTS; }

// Times every gather variant on a forward apply of zero sources and keeps
// the fastest (the other stages do not depend on the variant).
pim_status apply_autotune(pim_plan P, cudaStream_t s) {
    const PointsData& d = P->pts;
    if (d.N == 0) return PIM_OK;
    const size_t el = P->prec == PIM_FP64 ? sizeof(double) : sizeof(float);
    const size_t bytes = (size_t)d.N * el * (P->real_data ? 1 : 2);
    void *q = nullptr, *u = nullptr;
    pim_status st;
    if ((st = pim_alloc(P, &q, bytes)) != PIM_OK) return st;
    if ((st = pim_alloc(P, &u, bytes)) != PIM_OK) return st;
    PIM_CK(cudaMemsetAsync(q, 0, bytes, s));
    PIM_CK(cudaEventCreate(&P->tune_ev[0]));
    PIM_CK(cudaEventCreate(&P->tune_ev[1]));
    float best = 1e30f;
    int bestv = 0;
    const bool prof = P->prof_on;
    P->prof_on = false;
    const int64_t launches = P->launches;
    const int nvar = gather_variant_count(P);
    for (int v = 0; v < nvar; ++v) {
        P->gather_variant = v;
        if ((st = apply_run(P, q, u, 1, false, s)) != PIM_OK) return st;  // warm-up
        float tot = 0.f;
        for (int r = 0; r < 3; ++r) {
            if ((st = apply_run(P, q, u, 1, false, s)) != PIM_OK) return st;
            PIM_CK(cudaEventSynchronize(P->tune_ev[1]));
            float ms = 0.f;
            PIM_CK(cudaEventElapsedTime(&ms, P->tune_ev[0], P->tune_ev[1]));
            tot += ms;
        }
        if (tot < best) {
            best = tot;
            bestv = v;
        }
    }
    cudaEventDestroy(P->tune_ev[0]);
    cudaEventDestroy(P->tune_ev[1]);
    P->tune_ev[0] = P->tune_ev[1] = nullptr;
    P->prof_on = prof;
    P->launches = launches;
    P->gather_variant = bestv;
    pim_free(P, q, bytes);
    pim_free(P, u, bytes);
    return PIM_OK;
}

pim_status apply_run(pim_plan P, const void* q, void* u, int nrhs, bool adjoint, cudaStream_t s) {
    if (P->prec == PIM_FP64) return run_p<double>(P, q, u, nrhs, adjoint, s);
    return run_p<float>(P, q, u, nrhs, adjoint, s);
}
