// Point-dependent pre-processing (Sec. 3.2 and 3.3): binning into the grid's
// boxes by counting sort, per-point stencil data, and the near-pair
// correction list of Sec. 3.3 step 4 with its FP64 values.
#include <algorithm>
#include <cmath>
#include <vector>

#include <cuda_bf16.h>

#include <cub/device/device_radix_sort.cuh>

#include "pim_internal.cuh"

namespace {

constexpr double PI = 3.141592653589793238462643383279502884;

// exp(-j k R) / (4 pi R), k = k + j ki
__device__ __forceinline__ double2 G0(double R, double k, double ki) {
    double s, c;
    sincos(k * R, &s, &c);
    double a = 1.0 / (4.0 * PI * R);
    if (ki != 0.0) a *= exp(ki * R);
    return make_double2(c * a, -s * a);
}

// ------------------------------- exclusive scan ----------------------------
constexpr int SCAN_NT = 1024, SCAN_IPT = 4, SCAN_TILE = SCAN_NT * SCAN_IPT;

__device__ __forceinline__ long long block_scan_excl(long long v, long long* warp_tot, long long& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        long long t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        long long u = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += y;
        }
        warp_tot[lane] = u - t;  // exclusive warp offsets
        if (lane == 31) warp_tot[32] = u;
    }
    __syncthreads();
    total = warp_tot[32];
    const long long r = warp_tot[wid] + x - v;
    __syncthreads();
    return r;
}

__global__ void scan_block_sums(const int* in, long long n, long long* partial) {
    __shared__ long long wt[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_IPT;
    long long s = 0;
    for (int i = 0; i < SCAN_IPT; ++i)
        if (base + i < n) s += in[base + i];
    long long tot;
    block_scan_excl(s, wt, tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void scan_partials(long long* partial, long long nb, long long* total_out) {
    __shared__ long long wt[33];
    long long carry = 0;
    for (long long b0 = 0; b0 < nb; b0 += SCAN_NT) {
        const long long i = b0 + threadIdx.x;
        const long long v = i < nb ? partial[i] : 0;
        long long tot;
        const long long ex = block_scan_excl(v, wt, tot);
        if (i < nb) partial[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <typename OutT>
__global__ void scan_write(const int* in, long long n, const long long* partial, const long long* total, OutT* out) {
    __shared__ long long wt[33];
    const long long base = (long long)blockIdx.x * SCAN_TILE + threadIdx.x * SCAN_IPT;
    long long v[SCAN_IPT];
    long long s = 0;
    for (int i = 0; i < SCAN_IPT; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    long long tot;
    long long off = block_scan_excl(s, wt, tot) + partial[blockIdx.x];
    for (int i = 0; i < SCAN_IPT; ++i) {
        if (base + i < n) out[base + i] = (OutT)off;
        off += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (OutT)(*total);
}

// ------------------------------- binning -----------------------------------
struct BinArgs {
    double D[3], h[3];
    int nb[3];
    int p;
};

__global__ void keys_kernel(const double* xyz, long long N, BinArgs a, int* key, int* counts, int* status) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        int b[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
            const double x = xyz[3 * i + d];
            if (!(x >= 0.0 && x <= a.D[d])) ok = false;
            b[d] = box_of(x / a.h[d], a.nb[d], a.p);
        }
        if (!ok) atomicOr(status, 1);
        const int k = (b[2] * a.nb[1] + b[1]) * a.nb[0] + b[0];
        key[i] = k;
        atomicAdd(&counts[k], 1);
    }
}

__global__ void scatter_kernel(const int* key, long long N, const int* box_ptr, int* cursor, int* slot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const int k = key[i];
        const int pos = box_ptr[k] + atomicAdd(&cursor[k], 1);
        slot[pos] = (int)i;
    }
}

__global__ void nonempty_flags_kernel(const int* box_ptr, long long nboxes, int* flag) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nboxes;
         b += (long long)gridDim.x * blockDim.x)
        flag[b] = box_ptr[b + 1] > box_ptr[b] ? 1 : 0;
}

__global__ void box_slots_kernel(const int* flag, const int* pos, const int* box_ptr, long long nboxes, int* bslot,
                                 int* blist, int* bstart) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nboxes;
         b += (long long)gridDim.x * blockDim.x) {
        if (flag[b]) {
            bslot[b] = pos[b];
            blist[pos[b]] = (int)b;
            bstart[pos[b]] = box_ptr[b];
        } else {
            bslot[b] = -1;
        }
        if (b == nboxes - 1) bstart[pos[nboxes]] = box_ptr[nboxes];
    }
}

// first slot of each box row (box rows are runs of nb_x boxes along x)
__global__ void row_slots_kernel(const int* pos, long long nrows, int nbx, int* rsp) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r <= nrows;
         r += (long long)gridDim.x * blockDim.x)
        rsp[r] = pos[r * nbx];
}

// dense boxes (PIM_DENSE_MIN points or more) and their compact index
__global__ void dense_flags_kernel(const int* bstart, long long nne, int* flag) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nne; s += (long long)gridDim.x * blockDim.x)
        flag[s] = bstart[s + 1] - bstart[s] >= PIM_DENSE_MIN ? 1 : 0;
}

__global__ void dense_slots_kernel(const int* flag, const int* pos, long long nne, int* dix, int* dslot) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nne; s += (long long)gridDim.x * blockDim.x) {
        if (flag[s]) {
            dix[s] = pos[s];
            dslot[pos[s]] = (int)s;
        } else {
            dix[s] = -1;
        }
    }
}

// spread entries per box row: one for a dense box, one per point otherwise
__global__ void row_entries_kernel(const int* rsp, const int* bstart, const int* dix, long long nrows, int* cnt) {
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows; r += (long long)gridDim.x * blockDim.x) {
        int c = 0;
        for (int s = rsp[r]; s < rsp[r + 1]; ++s) c += dix[s] >= 0 ? 1 : bstart[s + 1] - bstart[s];
        cnt[r] = c;
    }
}

__global__ void row_fill_kernel(const int* rsp, const int* bstart, const int* dix, const int* blist, long long nrows,
                                int nb0, int nx, int p, const int* eptr, uint32_t* ent, uint16_t* esx) {
    const int lo = (p & 1) ? (p - 1) / 2 : p / 2;
    for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < nrows; r += (long long)gridDim.x * blockDim.x) {
        int e = eptr[r];
        for (int s = rsp[r]; s < rsp[r + 1]; ++s) {
            const int bx = blist[s] % nb0;
            const uint16_t sx = (uint16_t)min(max(bx - lo, 0), nx - 1 - p);
            if (dix[s] >= 0) {
                ent[e] = 0x80000000u | (uint32_t)dix[s];
                esx[e++] = sx;
            } else {
                for (int m = bstart[s]; m < bstart[s + 1]; ++m) {
                    ent[e] = (uint32_t)m;
                    esx[e++] = sx;
                }
            }
        }
    }
}

// order each box's points by caller index (deterministic layout)
__global__ void sort_boxes_kernel(const int* box_ptr, long long nboxes, int* slot) {
    for (long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x; b < nboxes;
         b += (long long)gridDim.x * blockDim.x) {
        const int lo = box_ptr[b], hi = box_ptr[b + 1];
        for (int i = lo + 1; i < hi; ++i) {
            const int v = slot[i];
            int j = i - 1;
            while (j >= lo && slot[j] > v) {
                slot[j + 1] = slot[j];
                --j;
            }
            slot[j + 1] = v;
        }
    }
}

struct PtArgs {
    double h[3], df[3];
    int n[3], nf[3], p, pf;
    int has_far;
};

__global__ void point_data_kernel(const double* xyz, const int* perm, long long N, PtArgs a, double* pos,
                                  uint32_t* ns, float* nt, double* ntd, uint32_t* fs, uint32_t* fo, float* ft,
                                  double* ftd) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const long long i = perm[m];
        int s[3], ss[3], so[3];
        for (int d = 0; d < 3; ++d) {
            const double x = xyz[3 * i + d];
            pos[3 * m + d] = x;
            const double u = x / a.h[d];
            s[d] = stencil_start(u, a.n[d], a.p);
            const double t = u - s[d];
            nt[3 * m + d] = (float)t;
            ntd[3 * m + d] = t;
            if (a.has_far) {
                const double uf = x / a.df[d];
                ss[d] = stencil_start(uf, a.nf[d], a.pf);
                const double uo = (x - 0.5 * a.df[d]) / a.df[d];
                so[d] = stencil_start(uo, a.nf[d], a.pf);
                ft[6 * m + d] = (float)(uf - ss[d]);
                ft[6 * m + 3 + d] = (float)(uo - so[d]);
                ftd[6 * m + d] = uf - ss[d];
                ftd[6 * m + 3 + d] = uo - so[d];
            }
        }
        ns[m] = pack3(s[0], s[1], s[2]);
        if (a.has_far) {
            fs[m] = pack3(ss[0], ss[1], ss[2]);
            fo[m] = pack3(so[0], so[1], so[2]);
        }
    }
}

// ------------------------------- near pairs --------------------------------
struct PairArgs {
    int nb[3], nL[3];
    int b, cube, p;
    int nimg;
    const int* img;     // nimg x 3
};

__device__ __forceinline__ int isqrt_floor(int r) {
    int g = (int)sqrt((double)r);
    while ((g + 1) * (g + 1) <= r) ++g;
    while (g * g > r) --g;
    return g;
}

// Visits every (image, source box row) of the correction region of the
// point in box B: calls f(image, box row, x0, x1, first sorted slot, end
// slot) for the boxes x0..x1 of that row that hold points.
template <typename F>
__device__ __forceinline__ void for_each_region_span(const PairArgs& a, const int* box_ptr, const int B[3], F f) {
    const int R = a.b + 1;
    for (int ii = 0; ii < a.nimg; ++ii) {
        int cb[3];
        for (int d = 0; d < 3; ++d) cb[d] = B[d] - a.img[3 * ii + d] * a.nL[d];
        for (int dz = -R; dz <= R; ++dz) {
            const int bz = cb[2] - dz;
            if (bz < 0 || bz >= a.nb[2]) continue;
            const int gz = abs(dz) > 1 ? abs(dz) - 1 : 0;
            for (int dy = -R; dy <= R; ++dy) {
                const int by = cb[1] - dy;
                if (by < 0 || by >= a.nb[1]) continue;
                const int gy = abs(dy) > 1 ? abs(dy) - 1 : 0;
                int xr;
                if (a.cube) {
                    if (abs(dz) > a.b || abs(dy) > a.b) continue;
                    xr = a.b;
                } else {
                    const int rem = a.b * a.b - gz * gz - gy * gy;
                    if (rem < 0) continue;
                    xr = isqrt_floor(rem) + 1;
                }
                int x0 = cb[0] - xr, x1 = cb[0] + xr;
                x0 = x0 < 0 ? 0 : x0;
                x1 = x1 > a.nb[0] - 1 ? a.nb[0] - 1 : x1;
                if (x0 > x1) continue;
                const long long row = ((long long)bz * a.nb[1] + by) * a.nb[0];
                const int lo = box_ptr[row + x0], hi = box_ptr[row + x1 + 1];
                if (hi > lo) f(ii, row, x0, x1, lo, hi);
            }
        }
    }
}

// The same with f(image, first sorted slot, end slot).
template <typename F>
__device__ __forceinline__ void for_each_region_row(const PairArgs& a, const int* box_ptr, const int B[3], F f) {
    for_each_region_span(a, box_ptr, B, [&](int ii, long long, int, int, int lo, int hi) { f(ii, lo, hi); });
}

// ------------------------------- list-free boxes ---------------------------
// A non-empty box whose correction work (its points times its region's
// points, the same for every point of the box) is at least thr is corrected
// list-free by every apply; its points' rows of the stored list are emptied.
__global__ void lf_flag_kernel(const int* bstart, long long nne, const int* rowlen, long long thr, int* flag,
                               unsigned long long* tot) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nne; s += (long long)gridDim.x * blockDim.x) {
        const int m0 = bstart[s], nA = bstart[s + 1] - m0;
        const long long work = (long long)nA * rowlen[m0];
        const bool f = thr > 0 && work >= thr;
        flag[s] = f ? 1 : 0;
        if (f) {
            atomicAdd(&tot[0], (unsigned long long)work);
            atomicAdd(&tot[1], (unsigned long long)nA);
        }
    }
}

__global__ void lf_list_kernel(const int* flag, const int* pos, long long nne, int* lfslot, int* lfmark) {
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < nne; s += (long long)gridDim.x * blockDim.x) {
        lfmark[s] = flag[s] ? pos[s] : -1;
        if (flag[s]) lfslot[pos[s]] = (int)s;
    }
}

// Region segments of every list-free box: runs of consecutive dense boxes
// (boxes with moments) inside one (image, box row) span, as (first slot, end
// slot, image | slot offset << 8, point offset), the offsets counted from the
// box's first segment.  The segments of the 27 boxes around the box (box
// offsets -1..1 on every axis after the image shift) come first: lfnear[j]
// receives the number of their points (the exact kernel sums these pairs
// with double-float coordinates).  The points of the region's other boxes
// stay in the stored rows of the box's points; sparse[j] receives their
// number; lfself[j] the offset of the box's own points in the list (-1 if
// the box has no moments: then they are not in it).  seg == nullptr: counts.
// sym (the exact kernel's list, FP32 plans): beyond the 27 boxes, a partner
// that is itself list-free, of a box with moments, is kept only by the box
// of the lower slot, whose segment carries the flag 128 in its image byte
// (the exact kernel then sums the pairs for both boxes); the other box drops it.
__global__ void lf_seg_kernel(PairArgs a, const int* box_ptr, const int* bslot, const int* blist, const int* bstart,
                              const int* dix, const int* lfslot, long long nlf, const int64_t* segptr, int* cnt,
                              int* sparse, int4* seg, int* lfself, int* lfnear, unsigned long long* pairs,
                              const int* lfmark = nullptr, int sym = 0) {
    int self_img = -1;
    for (int i = 0; i < a.nimg; ++i)
        if (a.img[3 * i] == 0 && a.img[3 * i + 1] == 0 && a.img[3 * i + 2] == 0) self_img = i;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nlf; j += (long long)gridDim.x * blockDim.x) {
        const int sA = lfslot[j];
        const int b = blist[sA];
        const int B[3] = {b % a.nb[0], (b / a.nb[0]) % a.nb[1], b / (a.nb[0] * a.nb[1])};
        int c = 0, soff = 0, ptoff = 0, nsp = 0, self = -1, nnear = 0;
        const int64_t o = seg ? segptr[j] : 0;
        for (int pass = 0; pass < 2; ++pass) {
            for_each_region_span(a, box_ptr, B, [&](int ii, long long row, int x0, int x1, int, int) {
                // offsets of the row from the image-shifted box
                const int by = (int)((row / a.nb[0]) % a.nb[1]), bz = (int)(row / ((long long)a.nb[0] * a.nb[1]));
                const int cx = B[0] - a.img[3 * ii] * a.nL[0];
                const bool nrow = abs(B[1] - a.img[3 * ii + 1] * a.nL[1] - by) <= 1 &&
                                  abs(B[2] - a.img[3 * ii + 2] * a.nL[2] - bz) <= 1;
                int fs = -1, ls = -1, two = 0;
                auto close = [&]() {
                    if (fs < 0) return;
                    if (ii == self_img && fs <= sA && sA <= ls) self = ptoff + (bstart[sA] - bstart[fs]);
                    if (seg) seg[o + c] = make_int4(fs, ls + 1, ii | (two << 7) | (soff << 8), ptoff);
                    soff += ls + 1 - fs;
                    ptoff += bstart[ls + 1] - bstart[fs];
                    ++c;
                    fs = ls = -1;
                };
                const bool asym = sym && pass == 1 && dix[sA] >= 0;
                for (int x = x0; x <= x1; ++x) {
                    const bool near = nrow && abs(x - cx) <= 1;
                    const int sl = bslot[row + x];
                    if (near != (pass == 0)) {
                        close();  // a box of the other pass breaks the run
                        continue;
                    }
                    if (sl < 0) continue;
                    if (dix[sl] >= 0) {
                        // (the box itself under another image stays one-way:
                        // both images of the pair are in its own list)
                        if (asym && lfmark[sl] >= 0 && sl != sA) {
                            if (sl < sA) {  // summed by that box for both
                                close();
                                continue;
                            }
                            if (fs >= 0 && !two) close();
                            two = 1;
                        } else if (two) {
                            close();
                            two = 0;
                        }
                        if (fs < 0) fs = sl;
                        ls = sl;
                    } else {
                        close();
                        nsp += bstart[sl + 1] - bstart[sl];
                    }
                }
                close();
            });
            if (pass == 0) nnear = ptoff;
        }
        if (!seg) {
            cnt[j] = c;
            sparse[j] = nsp;
        } else if (lfself) {
            lfself[j] = self;
            lfnear[j] = nnear;
            atomicAdd(pairs, (unsigned long long)(bstart[sA + 1] - bstart[sA]) * (unsigned long long)ptoff);
        }
    }
}

// the stored rows of a list-free box's points hold its sparse partners
__global__ void lf_rowlen_kernel(const int* lfslot, long long nlf, const int* bstart, const int* sparse, int* rowlen) {
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < nlf; j += (long long)gridDim.x * blockDim.x) {
        const int s = lfslot[j];
        for (int m = bstart[s]; m < bstart[s + 1]; ++m) rowlen[m] = sparse[j];
    }
}

// Box-centred local coordinates u - (B + 1/2 for odd p) in grid steps as an
// FP32 head (lfp, with the packed box's bits in w) and the FP32 rounding of
// the rest (lfl).  old != nullptr keeps the boxes of an earlier call (frozen
// topology).
__global__ void lf_point_kernel(const double* pos, long long N, double h0, double h1, double h2, int nb0, int nb1,
                                int nb2, int p, const float4* old, float4* lfp, float4* lfl) {
    const double h[3] = {h0, h1, h2};
    const int nb[3] = {nb0, nb1, nb2};
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        int B[3];
        if (old) unpack3(__float_as_uint(old[m].w), B[0], B[1], B[2]);
        float c[3], cl[3];
        for (int d = 0; d < 3; ++d) {
            const double u = pos[3 * m + d] / h[d];
            if (!old) B[d] = box_of(u, nb[d], p);
            const double cd = u - (B[d] + ((p & 1) ? 0.5 : 0.0));
            c[d] = (float)cd;
            cl[d] = (float)(cd - (double)c[d]);
        }
        lfp[m] = make_float4(c[0], c[1], c[2], __uint_as_float(pack3(B[0], B[1], B[2])));
        lfl[m] = make_float4(cl[0], cl[1], cl[2], 0.f);
    }
}

__global__ void pair_count_kernel(const double* pos, long long N, const double* hh, PairArgs a, const int* box_ptr,
                                  int* rowlen) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        int B[3];
        for (int d = 0; d < 3; ++d) B[d] = box_of(pos[3 * m + d] / hh[d], a.nb[d], a.p);
        long long cnt = 0;
        for_each_region_row(a, box_ptr, B, [&](int, int lo, int hi) { cnt += hi - lo; });
        rowlen[m] = (int)cnt;
    }
}

struct FillArgs {
    PairArgs pa;
    double h[3], D[3], k, ki;
    int p, R, W, self_img;
    const double2* gtab;   // g(e), e in [-R, R]^3, x fastest
    int corr_mode;
};

// d/dt of the Lagrange basis (product rule), runtime degree p
__device__ __forceinline__ void lagrange_dweights(int p, double t, double* dw) {
    for (int j = 0; j <= p; ++j) {
        double den = 1.0;
        for (int l = 0; l <= p; ++l)
            if (l != j) den *= (double)(j - l);
        double s = 0.0;
        for (int k = 0; k <= p; ++k) {
            if (k == j) continue;
            double pr = 1.0;
            for (int l = 0; l <= p; ++l)
                if (l != j && l != k) pr *= (t - l);
            s += pr;
        }
        dw[j] = s / den;
    }
}

// Correction value (Eq. er) for observer m, source n, image ii, before the
// phase: G0(r_m - r_n - i o L) [not for m = n, i = 0] minus the grid
// interaction sum_a sum_c w_m(a) w_n(c) g(a - c - i o (n-1)), the latter via
//   sum_e g(s_m - s_n - i o (n-1) + e) Cx(e_x) Cy(e_y) Cz(e_z),
//   Cd(e) = sum_{j - l = e} w_{m,d}[j] w_{n,d}[l].
// With GRAD, also its gradient with respect to r_m (the observer's weights
// replaced by their derivatives along one axis at a time).
template <bool GRAD>
__device__ double2 corr_value(const FillArgs& a, const double* pos, const uint32_t* ns, const double* ntd, long long m,
                              long long n, int ii, int* status, double2* grad) {
    const int p = a.p;
    int sm[3], sn[3];
    unpack3(ns[m], sm[0], sm[1], sm[2]);
    unpack3(ns[n], sn[0], sn[1], sn[2]);
    double C[3][2 * PIM_MAX_P + 1], dC[3][2 * PIM_MAX_P + 1];
    int base[3];
    for (int d = 0; d < 3; ++d) {
        double wm[PIM_MAX_P + 1], wn[PIM_MAX_P + 1], dwm[PIM_MAX_P + 1];
        lagrange_weights<double>(p, ntd[3 * m + d], wm);
        lagrange_weights<double>(p, ntd[3 * n + d], wn);
        if (GRAD) lagrange_dweights(p, ntd[3 * m + d], dwm);
        for (int e = 0; e <= 2 * p; ++e) C[d][e] = dC[d][e] = 0.0;
        for (int j = 0; j <= p; ++j)
            for (int l = 0; l <= p; ++l) {
                C[d][j - l + p] += wm[j] * wn[l];
                if (GRAD) dC[d][j - l + p] += dwm[j] * wn[l] / a.h[d];
            }
        base[d] = sm[d] - sn[d] - a.pa.img[3 * ii + d] * a.pa.nL[d];
        if (abs(base[d]) + p > a.R) {
            atomicOr(status, PIM_DEV_BOUNDS);
            if (GRAD)
                for (int k = 0; k < 3; ++k) grad[k] = make_double2(0.0, 0.0);
            return make_double2(0.0, 0.0);
        }
    }
    double2 grid = make_double2(0.0, 0.0), gg[3];
    for (int k = 0; k < 3; ++k) gg[k] = make_double2(0.0, 0.0);
    for (int ez = 0; ez <= 2 * p; ++ez) {
        double2 sy = make_double2(0.0, 0.0), dsyx = sy, dsyy = sy;
        for (int ey = 0; ey <= 2 * p; ++ey) {
            const double2* row =
                a.gtab + ((long long)(base[2] + ez - p + a.R) * a.W + (base[1] + ey - p + a.R)) * a.W + (base[0] - p + a.R);
            double2 sx = make_double2(0.0, 0.0), dsx = sx;
            for (int ex = 0; ex <= 2 * p; ++ex) {
                const double2 g = row[ex];
                sx.x += C[0][ex] * g.x;
                sx.y += C[0][ex] * g.y;
                if (GRAD) {
                    dsx.x += dC[0][ex] * g.x;
                    dsx.y += dC[0][ex] * g.y;
                }
            }
            sy.x += C[1][ey] * sx.x;
            sy.y += C[1][ey] * sx.y;
            if (GRAD) {
                dsyx.x += C[1][ey] * dsx.x;
                dsyx.y += C[1][ey] * dsx.y;
                dsyy.x += dC[1][ey] * sx.x;
                dsyy.y += dC[1][ey] * sx.y;
            }
        }
        grid.x += C[2][ez] * sy.x;
        grid.y += C[2][ez] * sy.y;
        if (GRAD) {
            gg[0].x += C[2][ez] * dsyx.x;
            gg[0].y += C[2][ez] * dsyx.y;
            gg[1].x += C[2][ez] * dsyy.x;
            gg[1].y += C[2][ez] * dsyy.y;
            gg[2].x += dC[2][ez] * sy.x;
            gg[2].y += dC[2][ez] * sy.y;
        }
    }
    double2 exact = make_double2(0.0, 0.0);
    double2 dex[3] = {exact, exact, exact};
    if (!(m == n && ii == a.self_img)) {
        double r[3], r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
            r[d] = pos[3 * m + d] - pos[3 * n + d] - a.pa.img[3 * ii + d] * a.D[d];
            r2 += r[d] * r[d];
        }
        if (r2 == 0.0) {  // two points coincide modulo the lattice: Eq. 1 is singular
            atomicOr(status, PIM_DEV_COINCIDENT);
            if (GRAD)
                for (int k = 0; k < 3; ++k) grad[k] = make_double2(0.0, 0.0);
            return make_double2(0.0, 0.0);
        }
        const double R = sqrt(r2);
        exact = G0(R, a.k, a.ki);
        if (GRAD) {
            // grad G0(R) = G0(R) (-jk - 1/R) r / R
            const double2 f = cmul(exact, make_double2(-1.0 / R + a.ki, -a.k));
            for (int d = 0; d < 3; ++d) dex[d] = make_double2(f.x * r[d] / R, f.y * r[d] / R);
        }
    }
    if (GRAD)
        for (int d = 0; d < 3; ++d) grad[d] = csub(dex[d], gg[d]);
    return csub(exact, grid);
}

// position derivatives of a value: FP64, or double-float splits in the same
// 16-byte slots when the apply accumulates in double-float
__device__ __forceinline__ void store_grad(const FillArgs& a, long long q, const double2* gr, double2* dval) {
    for (int k = 0; k < 3; ++k) {
        if (corr_df(a.corr_mode)) {
            const float rh = (float)gr[k].x, ih = (float)gr[k].y;
            reinterpret_cast<float4*>(dval)[3 * q + k] =
                make_float4(rh, (float)(gr[k].x - (double)rh), ih, (float)(gr[k].y - (double)ih));
        } else {
            dval[3 * q + k] = gr[k];
        }
    }
}

// bf16 bits of x, rounded to nearest even
__device__ __forceinline__ uint32_t bf16_bits(float x) { return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void store_value(const FillArgs& a, long long q, double2 d, double2* val, float4* valdf,
                                            float2* valf, uint32_t* valt) {
    val[q] = d;
    const float rh = (float)d.x, ih = (float)d.y;
    if (a.corr_mode == PIM_CORR_DOUBLE_FLOAT) {
        valdf[q] = make_float4(rh, (float)(d.x - (double)rh), ih, (float)(d.y - (double)ih));
    } else if (a.corr_mode == PIM_CORR_FP32) {
        valf[q] = make_float2(rh, ih);
    } else if (a.corr_mode == PIM_CORR_COMPACT) {
        // head rounded to FP32, tail (the FP64 remainder) rounded to bf16:
        // |d - head - tail| <= 2^-9 |tail| <= 2^-33 |d| per component
        valf[q] = make_float2(rh, ih);
        valt[q] = bf16_bits((float)(d.x - (double)rh)) | (bf16_bits((float)(d.y - (double)ih)) << 16);
    }
}

// One warp per point: first the row's columns (the region's points, image
// by image and box row by box row; for a point of a list-free box only the
// points of boxes without moments), then the values with the lanes over the
// whole row.
__global__ void pair_fill_kernel(const double* pos, const uint32_t* ns, const double* ntd, long long N, FillArgs a,
                                 const int* box_ptr, const int* bslot, const int* bstart, const int* dix,
                                 const int* lfmark, const int64_t* row_ptr, uint32_t* col, double2* val,
                                 float4* valdf, float2* valf, uint32_t* valt, double2* dval, int* status) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long m = warp; m < N; m += nwarps) {
        const long long r0 = row_ptr[m], r1 = row_ptr[m + 1];
        // every stored row of a box that is not list-free holds at least the
        // point itself
        if (r1 == r0) continue;
        int B[3];
        for (int d = 0; d < 3; ++d) B[d] = box_of(pos[3 * m + d] / a.h[d], a.pa.nb[d], a.pa.p);
        const long long bid = ((long long)B[2] * a.pa.nb[1] + B[1]) * a.pa.nb[0] + B[0];
        const bool lf = lfmark && lfmark[bslot[bid]] >= 0;
        long long off = r0;
        for_each_region_span(a.pa, box_ptr, B, [&](int ii, long long row, int x0, int x1, int lo, int hi) {
            if (!lf) {
                for (int n = lo + lane; n < hi; n += 32) col[off + (n - lo)] = (uint32_t)n | ((uint32_t)ii << PIM_COL_BITS);
                off += hi - lo;
                return;
            }
            for (int x = x0; x <= x1; ++x) {
                const int sl = bslot[row + x];
                if (sl < 0 || dix[sl] >= 0) continue;
                const int b0 = bstart[sl], b1 = bstart[sl + 1];
                for (int n = b0 + lane; n < b1; n += 32) col[off + (n - b0)] = (uint32_t)n | ((uint32_t)ii << PIM_COL_BITS);
                off += b1 - b0;
            }
        });
        if (off != r1) {
            if (lane == 0) atomicOr(status, PIM_DEV_BOUNDS);
            continue;
        }
        __syncwarp();
        for (long long q = r0 + lane; q < r1; q += 32) {
            const uint32_t c = col[q];
            const long long n = c & PIM_COL_MASK;
            const int ii = (int)(c >> PIM_COL_BITS);
            if (dval) {
                double2 gr[3];
                const double2 d = corr_value<true>(a, pos, ns, ntd, m, n, ii, status, gr);
                store_value(a, q, d, val, valdf, valf, valt);
                store_grad(a, q, gr, dval);
            } else {
                store_value(a, q, corr_value<false>(a, pos, ns, ntd, m, n, ii, status, nullptr), val, valdf, valf,
                            valt);
            }
        }
    }
}

// Recomputes the values of an existing correction list (frozen topology).
__global__ void pair_refill_kernel(const double* pos, const uint32_t* ns, const double* ntd, long long N, FillArgs a,
                                   const int64_t* row_ptr, const uint32_t* col, double2* val, float4* valdf,
                                   float2* valf, uint32_t* valt, double2* dval, int* status) {
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long m = warp; m < N; m += nwarps) {
        for (long long q = row_ptr[m] + lane; q < row_ptr[m + 1]; q += 32) {
            const uint32_t c = col[q];
            const long long n = c & PIM_COL_MASK;
            const int ii = (int)(c >> PIM_COL_BITS);
            if (dval) {
                double2 gr[3];
                const double2 d = corr_value<true>(a, pos, ns, ntd, m, n, ii, status, gr);
                store_value(a, q, d, val, valdf, valf, valt);
                store_grad(a, q, gr, dval);
            } else {
                store_value(a, q, corr_value<false>(a, pos, ns, ntd, m, n, ii, status, nullptr), val, valdf, valf,
                            valt);
            }
        }
    }
}

// Compact correction mode: reorders every row into [entries with |d| >
// 2^-split max_row |d|] [the others], each part in its former order, into
// fresh arrays, and sets nbig[m] to the size of the first part.  One warp
// per row: the row maximum, the count, then a ballot-ranked scatter.
__global__ void split_rows_kernel(long long N, const int64_t* row_ptr, int split, const uint32_t* col,
                                  const double2* val, const float2* valf, const uint32_t* valt, const double2* dval,
                                  uint32_t* col2, double2* val2, float2* valf2, uint32_t* valt2, double2* dval2,
                                  float2* dvalf2, int* nbig) {
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long m = warp; m < N; m += nwarps) {
        const long long r0 = row_ptr[m], r1 = row_ptr[m + 1];
        double mx = 0.0;  // largest |d|^2 of the row
        for (long long q = r0 + lane; q < r1; q += 32) {
            const double2 d = val[q];
            mx = fmax(mx, d.x * d.x + d.y * d.y);
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const double thr = split > 0 ? ldexp(mx, -2 * split) : -1.0;
        int nb = 0;
        for (long long q0 = r0; q0 < r1; q0 += 32) {
            const long long q = q0 + lane;
            bool big = false;
            if (q < r1) {
                const double2 d = val[q];
                big = d.x * d.x + d.y * d.y > thr;
            }
            nb += __popc(__ballot_sync(0xffffffffu, big));
        }
        long long ob = r0, os = r0 + nb;
        for (long long q0 = r0; q0 < r1; q0 += 32) {
            const long long q = q0 + lane;
            const bool in = q < r1;
            bool big = false;
            double2 d = make_double2(0.0, 0.0);
            if (in) {
                d = val[q];
                big = d.x * d.x + d.y * d.y > thr;
            }
            const unsigned mb = __ballot_sync(0xffffffffu, big), ms = __ballot_sync(0xffffffffu, in && !big);
            if (in) {
                const long long t = big ? ob + __popc(mb & below) : os + __popc(ms & below);
                col2[t] = col[q];
                val2[t] = d;
                valf2[t] = valf[q];
                valt2[t] = valt[q];
                if (dval)
                    for (int k = 0; k < 3; ++k) {
                        // double-float derivatives (re hi, re lo, im hi, im lo) and their heads
                        const double2 g = dval[3 * q + k];
                        dval2[3 * t + k] = g;
                        const float4 gf = *reinterpret_cast<const float4*>(&g);
                        dvalf2[3 * t + k] = make_float2(gf.x, gf.z);
                    }
            }
            ob += __popc(mb);
            os += __popc(ms);
        }
        if (lane == 0) nbig[m] = nb;
    }
}

// New positions with the stencil starts kept (frozen topology).
__global__ void point_update_kernel(const double* xyz, const int* perm, long long N, PtArgs a, const double* D,
                                    double* pos, const uint32_t* ns, float* nt, double* ntd, const uint32_t* fs,
                                    const uint32_t* fo, float* ft, double* ftd, int* status) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const long long i = perm[m];
        int s[3], ss[3], so[3];
        unpack3(ns[m], s[0], s[1], s[2]);
        if (a.has_far) {
            unpack3(fs[m], ss[0], ss[1], ss[2]);
            unpack3(fo[m], so[0], so[1], so[2]);
        }
        for (int d = 0; d < 3; ++d) {
            const double x = xyz[3 * i + d];
            if (!(x >= 0.0 && x <= D[d])) atomicOr(status, 8);
            pos[3 * m + d] = x;
            const double t = x / a.h[d] - s[d];
            nt[3 * m + d] = (float)t;
            ntd[3 * m + d] = t;
            if (a.has_far) {
                const double ts = x / a.df[d] - ss[d], to = (x - 0.5 * a.df[d]) / a.df[d] - so[d];
                ft[6 * m + d] = (float)ts;
                ft[6 * m + 3 + d] = (float)to;
                ftd[6 * m + d] = ts;
                ftd[6 * m + 3 + d] = to;
            }
        }
    }
}

__global__ void gtab_kernel(double2* gtab, int R, double h0, double h1, double h2, double k, double ki) {
    const int W = 2 * R + 1;
    const long long tot = (long long)W * W * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % W) - R, y = (int)((e / W) % W) - R, z = (int)(e / ((long long)W * W)) - R;
        const double r = sqrt((x * h0) * (x * h0) + (y * h1) * (y * h1) + (z * h2) * (z * h2));
        gtab[e] = r > 0.0 ? G0(r, k, ki) : make_double2(0.0, 0.0);
    }
}

// far cell (stencil start, x fastest) of every point and its index
__global__ void far_key_kernel(const uint32_t* fst, long long N, int nf0, int nf1, int* key, int* idx) {
    for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
        const uint32_t v = fst[m];
        const int x = (int)(v & 1023u), y = (int)((v >> 10) & 1023u), z = (int)((v >> 20) & 1023u);
        key[m] = (z * nf1 + y) * nf0 + x;
        idx[m] = (int)m;
    }
}

template <typename OutT>
pim_status scan(pim_plan P, const int* in, OutT* out, long long n, cudaStream_t s) {
    const long long nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    long long* part = nullptr;
    pim_status st;
    if ((st = pim_alloc(P, (void**)&part, sizeof(long long) * (nb + 1))) != PIM_OK) return st;
    if (nb > 0) scan_block_sums<<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, part);
    scan_partials<<<1, SCAN_NT, 0, s>>>(part, nb, part + nb);
    if (nb > 0) scan_write<OutT><<<(unsigned)nb, SCAN_NT, 0, s>>>(in, n, part, part + nb, out);
    else {
        OutT z = 0;
        PIM_CK(cudaMemcpyAsync(out, &z, sizeof(OutT), cudaMemcpyHostToDevice, s));
    }
    PIM_CK(cudaGetLastError());
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, part, sizeof(long long) * (nb + 1));
    return PIM_OK;
}

FillArgs fill_args(pim_plan P, const PairArgs& pr) {
    FillArgs fa{};
    fa.pa = pr;
    for (int i = 0; i < 3; ++i) { fa.h[i] = P->h[i]; fa.D[i] = P->D[i]; }
    fa.k = P->k;
    fa.ki = P->ki;
    fa.p = P->p;
    fa.R = P->b + 2 + 2 * P->p;
    fa.W = 2 * fa.R + 1;
    fa.corr_mode = P->corr_mode;
    fa.self_img = -1;
    for (int i = 0; i < P->nimg; ++i)
        if (P->img[i][0] == 0 && P->img[i][1] == 0 && P->img[i][2] == 0) fa.self_img = i;
    return fa;
}

}  // namespace

// Chooses the list-free boxes (lf_flag_kernel), empties their rows in
// rowlen, and builds their region segments, box-centred coordinates and the
// grid-kernel table of the local grid.
static pim_status lf_classify(pim_plan P, int* rowlen, const PairArgs& pr, cudaStream_t s) {
    PointsData& d = P->pts;
    d.nlf = d.nseg = d.lf_points = d.lf_pairs = 0;
    const long long nne = d.nne;
    if (P->lf_min_work <= 0 || d.N == 0 || nne == 0 || !lf_geom(P).EX) return PIM_OK;
    pim_status st;
    int *flag = nullptr, *pos = nullptr;
    unsigned long long* tot = nullptr;
    if ((st = pim_alloc(P, (void**)&flag, (size_t)nne * sizeof(int))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&pos, (size_t)(nne + 1) * sizeof(int))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&tot, 2 * sizeof(unsigned long long))) != PIM_OK) return st;
    PIM_CK(cudaMemsetAsync(tot, 0, 2 * sizeof(unsigned long long), s));
    lf_flag_kernel<<<1024, 256, 0, s>>>(d.bstart, nne, rowlen, P->lf_min_work, flag, tot);
    PIM_CK(cudaGetLastError());
    if ((st = scan<int>(P, flag, pos, nne, s)) != PIM_OK) return st;
    int nlf = 0;
    unsigned long long ht[2] = {0, 0};
    PIM_CK(cudaMemcpy(&nlf, pos + nne, sizeof(int), cudaMemcpyDeviceToHost));
    PIM_CK(cudaMemcpy(ht, tot, sizeof(ht), cudaMemcpyDeviceToHost));
    if (nlf > 0) {
        if ((st = pim_alloc(P, (void**)&d.lfslot, (size_t)nlf * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.lfmark, (size_t)nne * sizeof(int))) != PIM_OK) return st;
        lf_list_kernel<<<1024, 256, 0, s>>>(flag, pos, nne, d.lfslot, d.lfmark);
        PIM_CK(cudaGetLastError());
        int* cnt = flag;      // reuse (nlf <= nne)
        int* sparse = pos;    // reuse
        const unsigned nb = (unsigned)std::min<long long>((nlf + 127) / 128, 152 * 16);
        lf_seg_kernel<<<nb, 128, 0, s>>>(pr, d.box_ptr, d.bslot, d.blist, d.bstart, d.dix, d.lfslot, nlf, nullptr,
                                         cnt, sparse, nullptr, nullptr, nullptr, nullptr);
        PIM_CK(cudaGetLastError());
        lf_rowlen_kernel<<<nb, 128, 0, s>>>(d.lfslot, nlf, d.bstart, sparse, rowlen);
        PIM_CK(cudaGetLastError());
        if ((st = pim_alloc(P, (void**)&d.segptr, (size_t)(nlf + 1) * sizeof(int64_t))) != PIM_OK) return st;
        if ((st = scan<int64_t>(P, cnt, d.segptr, nlf, s)) != PIM_OK) return st;
        int64_t nseg = 0;
        PIM_CK(cudaMemcpy(&nseg, d.segptr + nlf, sizeof(int64_t), cudaMemcpyDeviceToHost));
        if ((st = pim_alloc(P, (void**)&d.seg, (size_t)nseg * sizeof(int4))) != PIM_OK) return st;
        d.nseg = nseg;
        if ((st = pim_alloc(P, (void**)&d.lfself, (size_t)nlf * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.lfnear, (size_t)nlf * sizeof(int))) != PIM_OK) return st;
        PIM_CK(cudaMemsetAsync(tot, 0, sizeof(unsigned long long), s));
        lf_seg_kernel<<<nb, 128, 0, s>>>(pr, d.box_ptr, d.bslot, d.blist, d.bstart, d.dix, d.lfslot, nlf, d.segptr,
                                         nullptr, nullptr, d.seg, d.lfself, d.lfnear, tot);
        PIM_CK(cudaGetLastError());
        if ((st = pim_alloc(P, (void**)&d.lfp, (size_t)d.N * sizeof(float4))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.lfl, (size_t)d.N * sizeof(float4))) != PIM_OK) return st;
        lf_point_kernel<<<1024, 256, 0, s>>>(d.pos, d.N, P->h[0], P->h[1], P->h[2], P->nb[0], P->nb[1], P->nb[2], P->p,
                                             nullptr, d.lfp, d.lfl);
        PIM_CK(cudaGetLastError());
        if ((st = lf_build_table(P, s)) != PIM_OK) return st;
        PIM_CK(cudaMemcpy(ht, tot, sizeof(unsigned long long), cudaMemcpyDeviceToHost));  // the exact pairs
        if (P->prec == PIM_FP32_MIXED) {
            // the exact kernel's list with the pairs of two list-free boxes once
            int* xcnt = nullptr;
            if ((st = pim_alloc(P, (void**)&xcnt, (size_t)nlf * sizeof(int))) != PIM_OK) return st;
            lf_seg_kernel<<<nb, 128, 0, s>>>(pr, d.box_ptr, d.bslot, d.blist, d.bstart, d.dix, d.lfslot, nlf, nullptr,
                                             xcnt, sparse, nullptr, nullptr, nullptr, nullptr, d.lfmark, 1);
            PIM_CK(cudaGetLastError());
            if ((st = pim_alloc(P, (void**)&d.xsegptr, (size_t)(nlf + 1) * sizeof(int64_t))) != PIM_OK) return st;
            if ((st = scan<int64_t>(P, xcnt, d.xsegptr, nlf, s)) != PIM_OK) return st;
            int64_t nx = 0;
            PIM_CK(cudaMemcpy(&nx, d.xsegptr + nlf, sizeof(int64_t), cudaMemcpyDeviceToHost));
            if ((st = pim_alloc(P, (void**)&d.xseg, (size_t)std::max<int64_t>(nx, 1) * sizeof(int4))) != PIM_OK)
                return st;
            d.nxseg = nx;
            lf_seg_kernel<<<nb, 128, 0, s>>>(pr, d.box_ptr, d.bslot, d.blist, d.bstart, d.dix, d.lfslot, nlf, d.xsegptr,
                                             nullptr, nullptr, d.xseg, nullptr, nullptr, nullptr, d.lfmark, 1);
            PIM_CK(cudaGetLastError());
            PIM_CK(cudaStreamSynchronize(s));
            pim_free(P, xcnt, (size_t)nlf * sizeof(int));
        }
    }
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, flag, (size_t)nne * sizeof(int));
    pim_free(P, pos, (size_t)(nne + 1) * sizeof(int));
    pim_free(P, tot, 2 * sizeof(unsigned long long));
    d.nlf = nlf;
    d.lf_pairs = (int64_t)ht[0];
    d.lf_points = (int64_t)ht[1];
    if (nlf > 0 && (st = lf_tc_prepare(P, s)) != PIM_OK) return st;
    return PIM_OK;
}

// New positions for the current points with the discrete structure kept.
// Splits every row of a compact-mode list (split_rows_kernel) out of place.
static pim_status split_rows(pim_plan P, cudaStream_t s) {
    PointsData& d = P->pts;
    pim_status st;
    const int64_t N = d.N, nnz = d.nnz;
    if (!d.nbig && (st = pim_alloc(P, (void**)&d.nbig, (size_t)std::max<int64_t>(1, N) * sizeof(int))) != PIM_OK)
        return st;
    if (N == 0) return PIM_OK;
    if (nnz == 0) {
        PIM_CK(cudaMemsetAsync(d.nbig, 0, (size_t)N * sizeof(int), s));
        return PIM_OK;
    }
    uint32_t *col2 = nullptr, *valt2 = nullptr;
    double2 *val2 = nullptr, *dval2 = nullptr;
    float2 *valf2 = nullptr, *dvalf2 = nullptr;
    if ((st = pim_alloc(P, (void**)&col2, nnz * sizeof(uint32_t))) != PIM_OK ||
        (st = pim_alloc(P, (void**)&val2, nnz * sizeof(double2))) != PIM_OK ||
        (st = pim_alloc(P, (void**)&valf2, nnz * sizeof(float2))) != PIM_OK ||
        (st = pim_alloc(P, (void**)&valt2, nnz * sizeof(uint32_t))) != PIM_OK ||
        (d.dval && (st = pim_alloc(P, (void**)&dval2, 3 * nnz * sizeof(double2))) != PIM_OK) ||
        (d.dval && (st = pim_alloc(P, (void**)&dvalf2, 3 * nnz * sizeof(float2))) != PIM_OK)) {
        pim_free(P, col2, nnz * sizeof(uint32_t));
        pim_free(P, val2, nnz * sizeof(double2));
        pim_free(P, valf2, nnz * sizeof(float2));
        pim_free(P, valt2, nnz * sizeof(uint32_t));
        pim_free(P, dval2, 3 * nnz * sizeof(double2));
        return st;
    }
    split_rows_kernel<<<152 * 16, 256, 0, s>>>(N, d.row_ptr, P->corr_split, d.col, d.val, d.valf, d.valt, d.dval, col2,
                                               val2, valf2, valt2, dval2, dvalf2, d.nbig);
    PIM_CK(cudaGetLastError());
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, d.col, nnz * sizeof(uint32_t));
    pim_free(P, d.val, nnz * sizeof(double2));
    pim_free(P, d.valf, nnz * sizeof(float2));
    pim_free(P, d.valt, nnz * sizeof(uint32_t));
    pim_free(P, d.dval, 3 * nnz * sizeof(double2));
    pim_free(P, d.dvalf, 3 * nnz * sizeof(float2));
    d.col = col2;
    d.val = val2;
    d.valf = valf2;
    d.valt = valt2;
    d.dval = dval2;
    d.dvalf = dvalf2;
    return PIM_OK;
}

pim_status points_update(pim_plan P, const double* xyz, cudaStream_t s) {
    PointsData& d = P->pts;
    const long long N = d.N;
    pim_status st;
    PIM_CK(cudaMemsetAsync(P->dstatus, 0, sizeof(int), s));
    double* dD = nullptr;
    if ((st = pim_alloc(P, (void**)&dD, sizeof(double) * 3)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(dD, P->D, sizeof(double) * 3, cudaMemcpyHostToDevice, s));
    PtArgs pa{};
    for (int i = 0; i < 3; ++i) {
        pa.h[i] = P->h[i]; pa.df[i] = P->df[i]; pa.n[i] = P->n[i]; pa.nf[i] = P->nf[i];
    }
    pa.p = P->p;
    pa.pf = P->pf;
    pa.has_far = P->has_far ? 1 : 0;
    if (N > 0)
        point_update_kernel<<<1024, 256, 0, s>>>(xyz, d.perm, N, pa, dD, d.pos, d.ns, d.nt, d.ntd, d.fs, d.fo, d.ft,
                                                 d.ftd, P->dstatus);
    if (N > 0 && d.lfp)
        lf_point_kernel<<<1024, 256, 0, s>>>(d.pos, N, P->h[0], P->h[1], P->h[2], P->nb[0], P->nb[1], P->nb[2], P->p,
                                             d.lfp, d.lfp, d.lfl);
    PIM_CK(cudaGetLastError());
    int hstat = 0;
    PIM_CK(cudaMemcpyAsync(&hstat, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, dD, sizeof(double) * 3);
    if (hstat) {
        pim_set_error("a point lies outside the closed cell [0, D]");
        return PIM_ERR_OUT_OF_CELL;
    }
    int* dimg = nullptr;
    if ((st = pim_alloc(P, (void**)&dimg, sizeof(int) * 3 * P->nimg)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(dimg, P->img, sizeof(int) * 3 * P->nimg, cudaMemcpyHostToDevice, s));
    PairArgs pr{};
    for (int i = 0; i < 3; ++i) { pr.nb[i] = P->nb[i]; pr.nL[i] = P->n[i] - 1; }
    pr.b = P->b;
    pr.cube = P->cube;
    pr.p = P->p;
    pr.nimg = P->nimg;
    pr.img = dimg;
    FillArgs fa = fill_args(P, pr);
    double2* gtab = nullptr;
    const size_t gsz = (size_t)fa.W * fa.W * fa.W * sizeof(double2);
    if ((st = pim_alloc(P, (void**)&gtab, gsz)) != PIM_OK) return st;
    gtab_kernel<<<256, 256, 0, s>>>(gtab, fa.R, P->h[0], P->h[1], P->h[2], P->k, P->ki);
    fa.gtab = gtab;
    if (N > 0 && d.nnz > 0)
        pair_refill_kernel<<<152 * 16, 256, 0, s>>>(d.pos, d.ns, d.ntd, N, fa, d.row_ptr, d.col, d.val, d.valdf,
                                                     d.valf, d.valt, d.dval, P->dstatus);
    PIM_CK(cudaGetLastError());
    PIM_CK(cudaMemcpyAsync(&hstat, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, gtab, gsz);
    pim_free(P, dimg, sizeof(int) * 3 * P->nimg);
    if (hstat & PIM_DEV_COINCIDENT) {
        pim_set_error("two points coincide (modulo the lattice): the periodic sum is singular");
        return PIM_ERR_ARG;
    }
    if (hstat) {
        pim_set_error("internal bounds check tripped while updating the correction values");
        return PIM_ERR_DEVICE;
    }
    if (P->corr_mode == PIM_CORR_COMPACT) return split_rows(P, s);
    return PIM_OK;
}

void points_free(pim_plan P) {
    lf_tc_free(P);
    PointsData& d = P->pts;
    const size_t N = (size_t)d.N;
    pim_free(P, d.perm, N * sizeof(int));
    pim_free(P, d.pos, 3 * N * sizeof(double));
    pim_free(P, d.ns, N * sizeof(uint32_t));
    pim_free(P, d.nt, 3 * N * sizeof(float));
    pim_free(P, d.ntd, 3 * N * sizeof(double));
    pim_free(P, d.fs, N * sizeof(uint32_t));
    pim_free(P, d.fo, N * sizeof(uint32_t));
    pim_free(P, d.fperm_s, d.fperm_s ? N * sizeof(int) : 0);
    pim_free(P, d.fperm_o, d.fperm_o ? N * sizeof(int) : 0);
    d.fperm_s = d.fperm_o = nullptr;
    pim_free(P, d.ft, 6 * N * sizeof(float));
    pim_free(P, d.ftd, 6 * N * sizeof(double));
    const size_t nboxes = (size_t)P->nb[0] * P->nb[1] * P->nb[2];
    pim_free(P, d.box_ptr, (nboxes + 1) * sizeof(int));
    pim_free(P, d.bslot, nboxes * sizeof(int));
    pim_free(P, d.blist, (size_t)std::max<int64_t>(1, d.nne) * sizeof(int));
    pim_free(P, d.bstart, (size_t)(d.nne + 1) * sizeof(int));
    pim_free(P, d.rsp, (size_t)(d.nrows + 1) * sizeof(int));
    pim_free(P, d.dslot, (size_t)std::max<int64_t>(1, d.nd) * sizeof(int));
    pim_free(P, d.eptr, (size_t)(d.nrows + 1) * sizeof(int));
    pim_free(P, d.ent, (size_t)std::max<int64_t>(1, d.ne) * sizeof(uint32_t));
    pim_free(P, d.esx, (size_t)std::max<int64_t>(1, d.ne) * sizeof(uint16_t));
    {
        const size_t np3 = (size_t)(P->p + 1) * (P->p + 1) * (P->p + 1);
        const size_t ge = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
        pim_free(P, d.mom, (size_t)std::max<int64_t>(1, d.nd) * np3 * ge);
    }
    pim_free(P, d.row_ptr, (N + 1) * sizeof(int64_t));
    pim_free(P, d.col, d.nnz * sizeof(uint32_t));
    pim_free(P, d.val, d.nnz * sizeof(double2));
    pim_free(P, d.valdf, d.nnz * sizeof(float4));
    pim_free(P, d.valf, d.nnz * sizeof(float2));
    pim_free(P, d.valt, d.nnz * sizeof(uint32_t));
    pim_free(P, d.dval, 3 * d.nnz * sizeof(double2));
    pim_free(P, d.dvalf, 3 * d.nnz * sizeof(float2));
    pim_free(P, d.nbig, (size_t)std::max<int64_t>(1, d.N) * sizeof(int));
    pim_free(P, d.dix, (size_t)std::max<int64_t>(1, d.nne) * sizeof(int));
    pim_free(P, d.lfslot, (size_t)d.nlf * sizeof(int));
    pim_free(P, d.lfself, (size_t)d.nlf * sizeof(int));
    pim_free(P, d.lfnear, (size_t)d.nlf * sizeof(int));
    pim_free(P, d.lfl, d.lfl ? N * sizeof(float4) : 0);
    pim_free(P, d.lfmark, (size_t)(d.lfmark ? d.nne : 0) * sizeof(int));
    pim_free(P, d.segptr, (size_t)(d.nlf + 1) * sizeof(int64_t));
    pim_free(P, d.seg, (size_t)d.nseg * sizeof(int4));
    pim_free(P, d.xsegptr, d.xsegptr ? (size_t)(d.nlf + 1) * sizeof(int64_t) : 0);
    pim_free(P, d.xseg, d.xseg ? (size_t)std::max<int64_t>(d.nxseg, 1) * sizeof(int4) : 0);
    d.xsegptr = nullptr;
    d.xseg = nullptr;
    d.nxseg = 0;
    pim_free(P, d.lfp, N * sizeof(float4));
    if (d.lfg) {
        const LfGeom G = lf_geom(P);
        const size_t H1 = G.H + 1;
        pim_free(P, d.lfg, H1 * H1 * H1 * (P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2)));
    }
    d = PointsData{};
}

pim_status points_build(pim_plan P, int64_t N, const double* xyz, cudaStream_t s) {
    PointsData& d = P->pts;
    pim_status st;
    const long long nboxes = (long long)P->nb[0] * P->nb[1] * P->nb[2];
    int *key = nullptr, *counts = nullptr, *cursor = nullptr;
    if ((st = pim_alloc(P, (void**)&key, N * sizeof(int))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&counts, nboxes * sizeof(int))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&cursor, nboxes * sizeof(int))) != PIM_OK) return st;
    PIM_CK(cudaMemsetAsync(counts, 0, nboxes * sizeof(int), s));
    PIM_CK(cudaMemsetAsync(cursor, 0, nboxes * sizeof(int), s));
    PIM_CK(cudaMemsetAsync(P->dstatus, 0, sizeof(int), s));
    BinArgs ba{};
    for (int i = 0; i < 3; ++i) { ba.D[i] = P->D[i]; ba.h[i] = P->h[i]; ba.nb[i] = P->nb[i]; }
    ba.p = P->p;
    d.N = N;
    if (N > 0) keys_kernel<<<1024, 256, 0, s>>>(xyz, N, ba, key, counts, P->dstatus);
    PIM_CK(cudaGetLastError());
    int hstat = 0;
    PIM_CK(cudaMemcpyAsync(&hstat, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIM_CK(cudaStreamSynchronize(s));
    if (hstat) {
        pim_free(P, key, N * sizeof(int));
        pim_free(P, counts, nboxes * sizeof(int));
        pim_free(P, cursor, nboxes * sizeof(int));
        d.N = 0;
        pim_set_error("a point lies outside the closed cell [0, D]");
        return PIM_ERR_OUT_OF_CELL;
    }
    if ((st = pim_alloc(P, (void**)&d.box_ptr, (nboxes + 1) * sizeof(int))) != PIM_OK) return st;
    if ((st = scan<int>(P, counts, d.box_ptr, nboxes, s)) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.perm, N * sizeof(int))) != PIM_OK) return st;
    if (N > 0) {
        scatter_kernel<<<1024, 256, 0, s>>>(key, N, d.box_ptr, cursor, d.perm);
        sort_boxes_kernel<<<(unsigned)((nboxes + 255) / 256), 256, 0, s>>>(d.box_ptr, nboxes, d.perm);
    }
    PIM_CK(cudaGetLastError());
    // compact slots of the non-empty boxes (for the box-moment spread)
    {
        int* pos = nullptr;
        if ((st = pim_alloc(P, (void**)&pos, (nboxes + 1) * sizeof(int))) != PIM_OK) return st;
        nonempty_flags_kernel<<<1024, 256, 0, s>>>(d.box_ptr, nboxes, cursor);
        if ((st = scan<int>(P, cursor, pos, nboxes, s)) != PIM_OK) return st;
        int nne = 0;
        PIM_CK(cudaMemcpy(&nne, pos + nboxes, sizeof(int), cudaMemcpyDeviceToHost));
        d.nne = nne;
        if ((st = pim_alloc(P, (void**)&d.bslot, nboxes * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.blist, (size_t)std::max(1, nne) * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.bstart, (size_t)(nne + 1) * sizeof(int))) != PIM_OK) return st;
        box_slots_kernel<<<1024, 256, 0, s>>>(cursor, pos, d.box_ptr, nboxes, d.bslot, d.blist, d.bstart);
        PIM_CK(cudaGetLastError());
        // row slot pointers
        d.nrows = (long long)P->nb[1] * P->nb[2];
        if ((st = pim_alloc(P, (void**)&d.rsp, (d.nrows + 1) * sizeof(int))) != PIM_OK) return st;
        row_slots_kernel<<<256, 256, 0, s>>>(pos, d.nrows, P->nb[0], d.rsp);
        // dense boxes
        int *dix = nullptr, *dpos = nullptr;
        if ((st = pim_alloc(P, (void**)&dix, (size_t)std::max(1, nne) * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&dpos, (size_t)(nne + 1) * sizeof(int))) != PIM_OK) return st;
        if (nne > 0) dense_flags_kernel<<<1024, 256, 0, s>>>(d.bstart, nne, cursor);
        if ((st = scan<int>(P, cursor, dpos, nne, s)) != PIM_OK) return st;
        int nd = 0;
        PIM_CK(cudaMemcpy(&nd, dpos + nne, sizeof(int), cudaMemcpyDeviceToHost));
        d.nd = nd;
        if ((st = pim_alloc(P, (void**)&d.dslot, (size_t)std::max(1, nd) * sizeof(int))) != PIM_OK) return st;
        if (nne > 0) dense_slots_kernel<<<1024, 256, 0, s>>>(cursor, dpos, nne, dix, d.dslot);
        const size_t np3 = (size_t)(P->p + 1) * (P->p + 1) * (P->p + 1);
        const size_t ge = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
        if ((st = pim_alloc(P, &d.mom, (size_t)std::max(1, nd) * np3 * ge)) != PIM_OK) return st;
        // spread entries by box row
        if ((st = pim_alloc(P, (void**)&d.eptr, (d.nrows + 1) * sizeof(int))) != PIM_OK) return st;
        if (d.nrows > 0) row_entries_kernel<<<256, 256, 0, s>>>(d.rsp, d.bstart, dix, d.nrows, cursor);
        if ((st = scan<int>(P, cursor, d.eptr, d.nrows, s)) != PIM_OK) return st;
        int ne = 0;
        PIM_CK(cudaMemcpy(&ne, d.eptr + d.nrows, sizeof(int), cudaMemcpyDeviceToHost));
        d.ne = ne;
        if ((st = pim_alloc(P, (void**)&d.ent, (size_t)std::max(1, ne) * sizeof(uint32_t))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.esx, (size_t)std::max(1, ne) * sizeof(uint16_t))) != PIM_OK) return st;
        if (d.nrows > 0)
            row_fill_kernel<<<256, 256, 0, s>>>(d.rsp, d.bstart, dix, d.blist, d.nrows, P->nb[0], P->n[0], P->p, d.eptr,
                                                d.ent, d.esx);
        PIM_CK(cudaGetLastError());
        PIM_CK(cudaStreamSynchronize(s));
        d.dix = dix;  // kept: the list-free correction reads the dense boxes' moments
        pim_free(P, dpos, (size_t)(nne + 1) * sizeof(int));
        pim_free(P, pos, (nboxes + 1) * sizeof(int));
    }
    // per-point data in sorted order
    if ((st = pim_alloc(P, (void**)&d.pos, 3 * N * sizeof(double))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.ns, N * sizeof(uint32_t))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.nt, 3 * N * sizeof(float))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.ntd, 3 * N * sizeof(double))) != PIM_OK) return st;
    if (P->has_far) {
        if ((st = pim_alloc(P, (void**)&d.fs, N * sizeof(uint32_t))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.fo, N * sizeof(uint32_t))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.ft, 6 * N * sizeof(float))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.ftd, 6 * N * sizeof(double))) != PIM_OK) return st;
    }
    PtArgs pa{};
    for (int i = 0; i < 3; ++i) {
        pa.h[i] = P->h[i]; pa.df[i] = P->df[i]; pa.n[i] = P->n[i]; pa.nf[i] = P->nf[i];
    }
    pa.p = P->p;
    pa.pf = P->pf;
    pa.has_far = P->has_far ? 1 : 0;
    if (N > 0)
        point_data_kernel<<<1024, 256, 0, s>>>(xyz, d.perm, N, pa, d.pos, d.ns, d.nt, d.ntd, d.fs, d.fo, d.ft, d.ftd);
    PIM_CK(cudaGetLastError());
    if (P->has_far && N > 0) {
        // the far spread's point orders: by stencil start on each far grid
        // (a stable sort: points of one stencil stay in box order)
        int *kin = nullptr, *kout = nullptr, *vin = nullptr;
        void* tmp = nullptr;
        size_t tb = 0;
        const int cells = P->nf[0] * P->nf[1] * P->nf[2];
        int bits = 1;
        while ((1 << bits) < cells) ++bits;
        if ((st = pim_alloc(P, (void**)&d.fperm_s, N * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&d.fperm_o, N * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&kin, N * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&kout, N * sizeof(int))) != PIM_OK) return st;
        if ((st = pim_alloc(P, (void**)&vin, N * sizeof(int))) != PIM_OK) return st;
        PIM_CK(cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, d.fperm_s, (int)N, 0, bits, s));
        if ((st = pim_alloc(P, &tmp, tb)) != PIM_OK) return st;
        for (int side = 0; side < 2; ++side) {
            far_key_kernel<<<1024, 256, 0, s>>>(side == 0 ? d.fs : d.fo, N, P->nf[0], P->nf[1], kin, vin);
            PIM_CK(cudaGetLastError());
            size_t t2 = tb;
            PIM_CK(cub::DeviceRadixSort::SortPairs(tmp, t2, kin, kout, vin, side == 0 ? d.fperm_s : d.fperm_o, (int)N, 0,
                                                   bits, s));
        }
        PIM_CK(cudaStreamSynchronize(s));
        pim_free(P, tmp, tb);
        pim_free(P, kin, N * sizeof(int));
        pim_free(P, kout, N * sizeof(int));
        pim_free(P, vin, N * sizeof(int));
    }
    // near-pair list
    int* dimg = nullptr;
    if ((st = pim_alloc(P, (void**)&dimg, sizeof(int) * 3 * P->nimg)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(dimg, P->img, sizeof(int) * 3 * P->nimg, cudaMemcpyHostToDevice, s));
    double* dh = nullptr;
    if ((st = pim_alloc(P, (void**)&dh, sizeof(double) * 3)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(dh, P->h, sizeof(double) * 3, cudaMemcpyHostToDevice, s));
    PairArgs pr{};
    for (int i = 0; i < 3; ++i) { pr.nb[i] = P->nb[i]; pr.nL[i] = P->n[i] - 1; }
    pr.b = P->b;
    pr.cube = P->cube;
    pr.p = P->p;
    pr.nimg = P->nimg;
    pr.img = dimg;
    int* rowlen = key;  // reuse
    if (N > 0) pair_count_kernel<<<1024, 256, 0, s>>>(d.pos, N, dh, pr, d.box_ptr, rowlen);
    PIM_CK(cudaGetLastError());
    if ((st = lf_classify(P, rowlen, pr, s)) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.row_ptr, (N + 1) * sizeof(int64_t))) != PIM_OK) return st;
    if ((st = scan<int64_t>(P, rowlen, d.row_ptr, N, s)) != PIM_OK) return st;
    int64_t nnz = 0;
    PIM_CK(cudaMemcpy(&nnz, d.row_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost));
    d.nnz = nnz;
    if ((st = pim_alloc(P, (void**)&d.col, nnz * sizeof(uint32_t))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&d.val, nnz * sizeof(double2))) != PIM_OK) return st;
    if (P->corr_mode == PIM_CORR_DOUBLE_FLOAT)
        if ((st = pim_alloc(P, (void**)&d.valdf, nnz * sizeof(float4))) != PIM_OK) return st;
    if (P->corr_mode == PIM_CORR_FP32 || P->corr_mode == PIM_CORR_COMPACT)
        if ((st = pim_alloc(P, (void**)&d.valf, nnz * sizeof(float2))) != PIM_OK) return st;
    if (P->corr_mode == PIM_CORR_COMPACT)
        if ((st = pim_alloc(P, (void**)&d.valt, nnz * sizeof(uint32_t))) != PIM_OK) return st;
    if (P->with_gradient)
        if ((st = pim_alloc(P, (void**)&d.dval, 3 * nnz * sizeof(double2))) != PIM_OK) return st;
    // table of g over the offsets a correction can reach
    FillArgs fa = fill_args(P, pr);
    double2* gtab = nullptr;
    const size_t gsz = (size_t)fa.W * fa.W * fa.W * sizeof(double2);
    if ((st = pim_alloc(P, (void**)&gtab, gsz)) != PIM_OK) return st;
    gtab_kernel<<<256, 256, 0, s>>>(gtab, fa.R, P->h[0], P->h[1], P->h[2], P->k, P->ki);
    fa.gtab = gtab;
    if (N > 0 && nnz > 0)
        pair_fill_kernel<<<152 * 16, 256, 0, s>>>(d.pos, d.ns, d.ntd, N, fa, d.box_ptr, d.bslot, d.bstart, d.dix,
                                                   d.lfmark, d.row_ptr, d.col, d.val, d.valdf, d.valf, d.valt, d.dval,
                                                   P->dstatus);
    PIM_CK(cudaGetLastError());
    if ((st = lf_check(P, s)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(&hstat, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, gtab, gsz);
    pim_free(P, dimg, sizeof(int) * 3 * P->nimg);
    pim_free(P, dh, sizeof(double) * 3);
    pim_free(P, key, N * sizeof(int));
    pim_free(P, counts, nboxes * sizeof(int));
    pim_free(P, cursor, nboxes * sizeof(int));
    if (hstat & PIM_DEV_COINCIDENT) {
        pim_set_error("two points coincide (modulo the lattice): the periodic sum is singular");
        return PIM_ERR_ARG;
    }
    if (hstat) {
        pim_set_error("internal bounds check tripped while building the correction list");
        return PIM_ERR_DEVICE;
    }
    if (P->corr_mode == PIM_CORR_COMPACT) return split_rows(P, s);
    return PIM_OK;
}
