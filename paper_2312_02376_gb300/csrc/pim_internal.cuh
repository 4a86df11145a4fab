// Internal declarations of libpim: the plan, device helpers, kernel entry points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pim.h"

#define PIM_CK(call)                                                    \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) {                                        \
            pim_set_error(std::string(#call) + ": " + cudaGetErrorString(e_)); \
            return PIM_ERR_CUDA;                                        \
        }                                                               \
    } while (0)

void pim_set_error(const std::string& msg);

// Column word of the correction list: sorted source index in the low bits,
// near-image code above it.
constexpr int PIM_COL_BITS = 25;
constexpr uint32_t PIM_COL_MASK = (1u << PIM_COL_BITS) - 1u;
constexpr int PIM_MAX_IMAGES = 125;
// boxes with at least this many points are spread through their moments,
// the points of the others one by one
constexpr int PIM_DENSE_MIN = 4;
constexpr int PIM_MAX_P = 6;

// correction modes whose sums run in double-float on the FP32 pipes
__host__ __device__ constexpr bool corr_df(int mode) {
    return mode == PIM_CORR_DOUBLE_FLOAT || mode == PIM_CORR_COMPACT;
}

// device-side status flags (bit set)
enum { PIM_DEV_NOT_NEUTRAL = 1, PIM_DEV_BOUNDS = 2, PIM_DEV_COINCIDENT = 4, PIM_DEV_TIMEOUT = 8 };

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using cplx = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ cplx<T> mk(T re, T im) {
    cplx<T> c; c.x = re; c.y = im; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename T> __host__ __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }

// ---------------------------------------------------------------------------
// Lagrange weights (Sec. 3.2): w_j(t) = prod_{l != j} (t - l) / (j - l),
// j = 0..p, from prefix and suffix products of (t - l).
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ __forceinline__ void lagrange_weights(int p, T t, T* w) {
    T pre[PIM_MAX_P + 1], suf[PIM_MAX_P + 1];
    pre[0] = T(1);
    for (int j = 1; j <= p; ++j) pre[j] = pre[j - 1] * (t - T(j - 1));
    suf[p] = T(1);
    for (int j = p - 1; j >= 0; --j) suf[j] = suf[j + 1] * (t - T(j + 1));
    // denominator prod_{l != j} (j - l) = (-1)^{p-j} j! (p-j)!
    T fact[PIM_MAX_P + 1];
    fact[0] = T(1);
    for (int j = 1; j <= p; ++j) fact[j] = fact[j - 1] * T(j);
    for (int j = 0; j <= p; ++j) {
        T den = fact[j] * fact[p - j];
        if ((p - j) & 1) den = -den;
        w[j] = pre[j] * suf[j] / den;
    }
}

// Register-only selection w[j] for a runtime j < N (no local memory).
template <int N, typename T>
__host__ __device__ __forceinline__ T pick(const T* w, int j) {
    T r = w[0];
#pragma unroll
    for (int i = 1; i < N; ++i) r = (j == i) ? w[i] : r;
    return r;
}

// Lagrange weights for a runtime degree p <= PIM_MAX_P with fully unrolled,
// predicated loops (the array stays in registers).
template <typename T>
__host__ __device__ __forceinline__ void lagrange_weights_rt(int p, T t, T* w) {
    T pre[PIM_MAX_P + 1], suf[PIM_MAX_P + 1];
    pre[0] = T(1);
#pragma unroll
    for (int j = 1; j <= PIM_MAX_P; ++j) pre[j] = pre[j - 1] * (t - T(j - 1));
#pragma unroll
    for (int j = 0; j <= PIM_MAX_P; ++j) suf[j] = T(1);
#pragma unroll
    for (int j = PIM_MAX_P - 1; j >= 0; --j) suf[j] = (j + 1 <= p) ? suf[j + 1] * (t - T(j + 1)) : T(1);
#pragma unroll
    for (int j = 0; j <= PIM_MAX_P; ++j) {
        T den = T(1);
#pragma unroll
        for (int l = 0; l <= PIM_MAX_P; ++l)
            if (l != j && l <= p) den *= T(j - l);
        w[j] = j <= p ? pre[j] * suf[j] / den : T(0);
    }
}

// Stencil rule: even p: floor(u + 1/2) - p/2; odd p: floor(u) - (p-1)/2;
// clamped to [0, n-1-p].  Decided in FP64.
__host__ __device__ __forceinline__ int stencil_start(double u, int n, int p) {
    int s = (p & 1) ? (int)floor(u) - (p - 1) / 2 : (int)floor(u + 0.5) - p / 2;
    if (s < 0) s = 0;
    if (s > n - 1 - p) s = n - 1 - p;
    return s;
}

// Box of a coordinate: the cell of points that share one stencil.  Even p:
// the box centred on node floor(u + 1/2) (nb = n boxes); odd p: the grid
// cell floor(u) (nb = n-1 boxes).  u = x / h in FP64, as in stencil_start.
__host__ __device__ __forceinline__ int box_of(double u, int nb, int p) {
    int b = (p & 1) ? (int)floor(u) : (int)floor(u + 0.5);
    if (b < 0) b = 0;
    if (b > nb - 1) b = nb - 1;
    return b;
}

__host__ __device__ __forceinline__ uint32_t pack3(int a, int b, int c) {
    return (uint32_t)a | ((uint32_t)b << 10) | ((uint32_t)c << 20);
}
__host__ __device__ __forceinline__ void unpack3(uint32_t v, int& a, int& b, int& c) {
    a = v & 1023; b = (v >> 10) & 1023; c = (v >> 20) & 1023;
}

// ---------------------------------------------------------------------------
// FFT plan for one padded 3D grid: lengths L[d] (powers of two), the data
// lengths n[d] (<= L[d]) that are nonzero on input / kept on output.
// ---------------------------------------------------------------------------
struct FftGeom {
    int n[3];   // data nodes per axis
    int L[3];   // padded FFT length per axis
    // stored spectrum: along an axis in `fold` (bit d) the kernel is even, so
    // its spectrum is too and only frequencies 0..L/2 are kept (S = L/2 + 1)
    int fold = 0;
    int S[3] = {0, 0, 0};
};

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct PointsData {
    int64_t N = 0;
    int* perm = nullptr;          // sorted slot -> caller index
    double* pos = nullptr;        // sorted positions, 3N (x, y, z interleaved)
    uint32_t* ns = nullptr;       // near stencil starts, packed
    float* nt = nullptr;          // near local coordinates (FP32), 3N
    double* ntd = nullptr;        // near local coordinates (FP64), 3N
    uint32_t* fs = nullptr;       // far source-grid stencil starts, packed
    uint32_t* fo = nullptr;       // far observer-grid stencil starts, packed
    // the points (box order indices) sorted by their far stencil start on the
    // source and on the observer grid, for the far spread: runs of points that
    // share a stencil are summed in registers before one shared-memory addition
    int* fperm_s = nullptr;
    int* fperm_o = nullptr;
    float* ft = nullptr;          // far local coordinates, source grid then observer grid (6N)
    double* ftd = nullptr;        // same in FP64 (FP64 plans)
    int* box_ptr = nullptr;       // nboxes + 1
    int* bslot = nullptr;         // nboxes: compact index of a non-empty box, -1 if empty
    int* blist = nullptr;         // nne: box id of each non-empty box (box order)
    int* bstart = nullptr;        // nne + 1: first sorted point of each non-empty box
    int* rsp = nullptr;           // nrows + 1: first slot of each box row (y, z)
    long long nrows = 0;
    int64_t nne = 0;              // non-empty boxes
    int* dslot = nullptr;         // nd: slot of each dense box (PIM_DENSE_MIN points or more)
    int64_t nd = 0;
    int* eptr = nullptr;          // nrows + 1: first spread entry of each box row
    uint32_t* ent = nullptr;      // ne spread entries in box-row order: a dense box (bit 31 | dense
                                  // index) or, for the other boxes, each point (sorted index)
    uint16_t* esx = nullptr;      // ne: stencil start along x of each entry
    int64_t ne = 0;
    void* mom = nullptr;          // nd x (p+1)^3 moments of the dense boxes, complex<T> (apply scratch)
    int64_t* row_ptr = nullptr;   // N + 1
    uint32_t* col = nullptr;      // nnz
    double2* val = nullptr;       // nnz: G0 - G_grid (FP64)
    float4* valdf = nullptr;      // nnz: double-float split (re_hi, re_lo, im_hi, im_lo)
    float2* valf = nullptr;       // nnz: complex64 (FP32 mode), or the FP32 heads (compact mode)
    uint32_t* valt = nullptr;     // nnz: bf16 tails of re (low half) and im (high half), compact mode
    int* nbig = nullptr;          // N: compact mode, entries at the head of each row summed in double-float
    double2* dval = nullptr;      // 3 nnz: d/dr_m of the values (with_gradient)
    float2* dvalf = nullptr;      // 3 nnz: their FP32 heads (compact mode; read for a row's complex64 part)
    int64_t nnz = 0;
    int* dix = nullptr;           // nne: dense index of each non-empty box, -1 if not dense
    // list-free correction: observer boxes whose correction is recomputed by
    // every apply (exact sum over the region's points minus the region's grid
    // interaction through a local grid of box moments); their rows of the
    // stored list are empty
    int64_t nlf = 0;              // list-free observer boxes
    int* lfslot = nullptr;        // nlf: slot of each
    int* lfmark = nullptr;        // nne: list-free index of each non-empty box, -1 if stored
    int* lfself = nullptr;        // nlf: offset of the box's own points in its region list, -1 if absent
    int* lfnear = nullptr;        // nlf: points of the 27 surrounding boxes, first in the region list
    float4* lfl = nullptr;        // N: FP32 rounding of the rest of the box-centred coordinates
    int64_t* segptr = nullptr;    // nlf + 1: first region segment of each
    int4* seg = nullptr;          // nseg: (first slot, end slot, image | slot offset << 8, point offset)
    int64_t nseg = 0;
    float4* lfp = nullptr;        // N: box-centred local coordinates (grid steps) and the packed box (w bits)
    void* lfg = nullptr;          // (H+1)^3 grid kernel g(|e|) on the offsets of the local grid, plan precision
    // the exact kernel's list in FP32 plans: segments as seg, with the pairs of
    // two list-free boxes (beyond the 27 boxes) kept by the box of lower slot
    // only, flagged 128 in the image byte (summed there for both boxes)
    int64_t* xsegptr = nullptr;       // nlf + 1
    int4* xseg = nullptr;
    int64_t nxseg = 0;
    // grid part on the tensor cores (FP32 plans): the interior list-free boxes
    unsigned char* tcmask = nullptr;  // nlf: 1 if box j is handled there
    int* tcl = nullptr;               // ntc list-free indices
    int64_t ntc = 0;
    int tcKP = 0;                     // E^3 padded to a multiple of 32
    long long tcbatch = 0;            // boxes per batch
    float* tcA = nullptr;             // forward hi, lo, adjoint hi, lo: 4 x 256 x 2 tcKP
    float* tcB = nullptr;             // a batch's FP32 Q rows, tcbatch x 2 tcKP
    float* tcC = nullptr;             // tcbatch x 256 products
    int64_t lf_points = 0;        // points in list-free boxes
    int64_t lf_pairs = 0;         // (observer, source, image) pairs their correction sums per apply
};

// Geometry of the list-free correction's local grid (see listfree.cu): c =
// floor(p/2), R = b + 1 the box reach of the correction region, E = 2R + 2c +
// p + 1 nodes per axis, H = R + 2c + p the largest node offset.
struct LfGeom {
    int c, R, E, H, EX;           // EX: padded x-length of a local grid row (16 or 24), 0 if unsupported
    int nterm;                    // terms of the exact kernel's cos / sinc polynomials; 0: sincos
};
LfGeom lf_geom(const pim_plan_s* P);

struct pim_plan_s {
    // geometry and method parameters
    double D[3], h[3], k, k0[3], df[3];
    double ki = 0.0, k0i[3] = {0.0, 0.0, 0.0};  // imaginary parts of k and k0
    unsigned pmask = 0;
    int npd = 0;                  // number of periodic axes
    int n[3], nb[3], p, layers, b, cube, nf[3], pf, prec, corr_mode;
    bool npsp = false;
    bool real_data = false;
    double neutral_tol, series_tol;
    size_t mem_cap = 0, bytes = 0;
    int nimg = 0;
    int img[PIM_MAX_IMAGES][3];
    double2 phase[PIM_MAX_IMAGES];    // exp(-j k0.(i o L))
    double2 phase_adj[PIM_MAX_IMAGES];  // exp(-j conj(k0).(i o L)) (the adjoint's)
    // near spectrum and work grids
    FftGeom ng;
    void* spec = nullptr;         // [Lz][Ly][Lx] complex<T>, scaled by 1/(Lx Ly Lz)
    void* gA = nullptr;           // [nz][ny][nx]
    void* gB = nullptr;           // [nz][ny][Lx]
    void* gC = nullptr;           // [nz][Ly][Lx]
    // far zone
    bool has_far = false;
    FftGeom fg;
    double2* ftab = nullptr;      // (2nf-1)^3 table, x fastest
    double2* fspec = nullptr;     // [Lz][Ly][Lx] FP64 spectrum of the far table, scaled
    double2* fA = nullptr;        // far grid charges / potentials [nfz][nfy][nfx]
    double2* fB = nullptr;        // [nfz][nfy][Lx]
    double2* fC = nullptr;        // [nfz][Ly][Lx]
    void* fpart = nullptr;        // far spread partials [nchunk][nf^3] complex<T>
    int far_chunks = 0;
    bool far_window = false;      // far grid spread by z-windows (too large for per-CTA partials)
    // twiddles (cos, sin of 2 pi j / L) per padded length, FP32 and FP64 copies
    float2* tw32 = nullptr;       // concatenated tables, offsets per power of two
    double2* tw64 = nullptr;
    int tw_off[12];
    // points
    PointsData pts;
    void* qs = nullptr;           // sorted sources, complex<T>, N
    void* us = nullptr;           // staging for host pointers
    void* ufp = nullptr;          // far part of every point (sorted order), complex<T>, N (with a far zone)
    size_t stage_bytes = 0;
    void* hq = nullptr;           // device staging of caller buffers (host pointers)
    void* hu = nullptr;
    double* dsum = nullptr;       // FP64 scratch: [0..1] mean, [4..) reduction partials
    double2* dphase = nullptr;    // device copy of phase[], followed by its double-float split
    float4* dphasedf = nullptr;   // (re hi, re lo, im hi, im lo), inside the dphase allocation
    // the adjoint's image phases exp(-j conj(k0).(i o L)) (equal to phase[] for
    // a real k0), same layout, inside the same allocation
    double2* dphase_adj = nullptr;
    float4* dphasedf_adj = nullptr;
    int* dstatus = nullptr;
    // profiling ring (pim_set_profiling)
    static constexpr int PROF_RING = 512;
    bool prof_on = false;
    int prof_next = 0;             // applies recorded since the reset
    cudaEvent_t* prof_ev = nullptr;  // [PROF_RING][PIM_NUM_STAGES][2]
    unsigned short prof_mask[512];   // stages recorded per ring slot (bit per stage)
    int64_t launches = 0;
    int gather_variant = 0;       // launch shape of the gather kernel (autotuned)
    int force_variant = -1;       // >= 0: launch shape fixed by the options
    // grid potentials kept for pim_position_grad_reuse (with_gradient plans):
    // bit 1: gA and fU hold those of the last single-RHS forward apply; bit 2:
    // gD and fV those of the last single-RHS adjoint apply
    int pot_valid = 0;
    bool keep_off = false;        // an apply on borrowed scratch (pim_apply_noalloc) keeps nothing
    int corr_split = 10;          // compact mode: threshold 2^-corr_split of the row's largest |d|
    cudaEvent_t tune_ev[2] = {nullptr, nullptr};  // around the gather launch while autotuning
    void* qsall = nullptr;        // sorted sources of every right-hand side (multi-RHS correction)
    size_t qsall_bytes = 0;
    double* dmeans = nullptr;     // per-RHS means (neutral static case), 2 x 128
    bool no_multi = false;        // keep the fused per-RHS path (set by pim_apply_noalloc)
    int autotune = 1;
    int with_gradient = 0;
    int lf_tc = 1;                // list-free grid part on the tensor cores where it applies
    int lf_min_work = 0;          // list-free boxes: n_box x region points >= this (0: off)
    void* gD = nullptr;           // second full grid (adjoint potential of the gradient)
    void* gsrt = nullptr;         // sorted upstream gradient g, complex<T>, N
    double2* fD = nullptr;        // second far grid
    void* fU = nullptr;           // far potentials in plan precision (gradient)
    void* fV = nullptr;
    // streams and events
    cudaStream_t s_main = nullptr;  // the plan's own stream inside a batched graph
    cudaStream_t s_far = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // list-free boxes (one right-hand side): their exact part, then their grid
    // part once the spread has formed the box moments, run on their own
    // low-priority stream into ulf (sorted order), concurrently with the
    // spread, FFT and gather; ulf is added to the output after the gather
    cudaStream_t s_lf = nullptr;
    cudaEvent_t ev_lf_fork = nullptr, ev_lf_mom = nullptr, ev_lf_join = nullptr;
    void* ulf = nullptr;            // N x complex<T> (plans with list-free boxes)
    unsigned long long* lfnext = nullptr;  // box counters of the exact-part kernel: one per lane, + async
    // observer points (pim_set_points_observers): the last nobs of the point
    // set; sources [0, nsrc); padded right-hand sides and results, per-RHS means
    int64_t nsrc = 0, nobs = 0;
    void* obs_q = nullptr;
    void* obs_u = nullptr;
    size_t obs_bytes = 0;
    double* obs_means = nullptr;
    int obs_nmeans = 0;
    double plan_ms = 0, points_ms = 0;
    // extra lanes of a multi-RHS apply: right-hand side r runs its per-RHS
    // stages on lane r % nlanes, each lane with its own scratch and streams
    // (lane 0 is the plan's own scratch above)
    static constexpr int RHS_LANES = 4;
    struct Lane {
        void* qs = nullptr;
        void* gA = nullptr;
        void* gB = nullptr;
        void* gC = nullptr;
        void* mom = nullptr;
        void* fpart = nullptr;
        double2* fA = nullptr;
        double2* fB = nullptr;
        double2* fC = nullptr;
        void* ufp = nullptr;
        cudaStream_t sm = nullptr, sf = nullptr;
        cudaEvent_t fork = nullptr, join = nullptr, done = nullptr;
    } lane[RHS_LANES];
    int nlanes = 1;                // lanes allocated (1: none extra)
    cudaEvent_t lane_fork = nullptr;
};

// ---------------------------------------------------------------------------
// internal entry points (defined in the .cu files)
// ---------------------------------------------------------------------------
pim_status pim_alloc(pim_plan P, void** ptr, size_t bytes);
void pim_free(pim_plan P, void* ptr, size_t bytes);

// fft.cu
pim_status fft_make_twiddles(pim_plan P);
template <typename T>
pim_status fft3_conv(pim_plan P, const FftGeom& g, cplx<T>* A, cplx<T>* B, cplx<T>* C, const cplx<T>* spec,
                     bool conj_spec, cudaStream_t s);
template <typename T>
pim_status fft3_forward_full(pim_plan P, const FftGeom& g, cplx<T>* X, cplx<T>* tmp, cudaStream_t s);

// tables.cu
pim_status build_near_spectrum(pim_plan P, cudaStream_t s);
pim_status build_far_table(pim_plan P, cudaStream_t s);

// points.cu
pim_status points_build(pim_plan P, int64_t N, const double* xyz_dev, cudaStream_t s);
pim_status points_update(pim_plan P, const double* xyz_dev, cudaStream_t s);
void points_free(pim_plan P);

// profiling: record the start / stop event of a stage of the current apply
void prof_mark(pim_plan P, int stage, int which, cudaStream_t s);

// apply.cu
constexpr int PIM_RED_BLOCKS = 608;
pim_status apply_run(pim_plan P, const void* q, void* u, int nrhs, bool adjoint, cudaStream_t s);
pim_status apply_debug_spread(pim_plan P, void* out_dev, cudaStream_t s);
pim_status apply_autotune(pim_plan P, cudaStream_t s);
int far_stream_priority();  // the device's highest stream priority
int gather_variant_count(const pim_plan_s* P);
pim_status grad_run(pim_plan P, const void* q, const void* g, double* grad, int nrhs, cudaStream_t s,
                    bool reuse = false);
pim_status alloc_grad_buffers(pim_plan P);
pim_status apply_prepare(pim_plan P, int nrhs, bool adjoint);
pim_status lanes_prepare(pim_plan P, int nlanes);
void lanes_free(pim_plan P);

// observers.cu
void observers_free(pim_plan P);

// listfree.cu
pim_status lf_apply(pim_plan P, const void* qs, void* dst, int nrhs, int r, bool adj, bool sorted_out,
                    cudaStream_t s, int lane = 0);
pim_status lf_exact_async(pim_plan P, const void* qs, bool adj, cudaStream_t s);
pim_status lf_grid_async(pim_plan P, const void* qs, bool adj, cudaStream_t s);
pim_status lf_add(pim_plan P, void* dst, bool sorted_out, cudaStream_t s);
int lf_stream_priority();  // the device's lowest stream priority
pim_status lf_check(pim_plan P, cudaStream_t s);
pim_status lf_build_table(pim_plan P, cudaStream_t s);
pim_status lf_tc_prepare(pim_plan P, cudaStream_t s);  // after the list-free tables and nlf
void lf_tc_free(pim_plan P);

// batch.cu
void batch_forget(pim_plan P);
int pim_fft_len(int n);
