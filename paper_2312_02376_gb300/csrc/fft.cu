// Shared-memory Stockham FFT passes for the zero-padded grid convolution of
// Sec. 3.3 step 2 (and of the far-zone grid sum of Eq. 8).
//
// A CTA transforms B columns of length L held in shared memory as
// s[row * LD + col] (LD = B + 1).  Lanes run along columns, so every stage's
// shared-memory accesses by a warp are to consecutive words.  Each stage is a
// radix-R (8, 4 or 2) Stockham step in natural order:
//   v_r = x[j + r L/R], twiddled by W_{Ns R}^{r (j mod Ns)}, R-point DFT,
//   stored at (j / Ns) Ns R + (j mod Ns) + r Ns.
// Passes are pruned: a pass loads n_in rows (the rest are the zero padding)
// and stores n_keep rows, so the zero half of each axis is never read from
// or written to global memory.  The z pass multiplies by the spectrum
// between its forward and inverse transforms.
#include <cmath>

#include "pim_internal.cuh"

namespace {

constexpr int LMAX = 2048;  // twiddle table length

template <typename C, bool INV> __device__ __forceinline__ C mul_mj(C a) {
    // forward: multiply by -j; inverse: by +j
    C r;
    if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

template <typename T, bool INV> __device__ __forceinline__ void dft2(cplx<T>* v) {
    cplx<T> a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
}

template <typename T, bool INV> __device__ __forceinline__ void dft4(cplx<T>* v) {
    cplx<T> a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    cplx<T> a2 = cadd(v[1], v[3]), a3 = mul_mj<cplx<T>, INV>(csub(v[1], v[3]));
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3);
    v[3] = csub(a1, a3);
}

template <typename T, bool INV> __device__ __forceinline__ void dft8(cplx<T>* v) {
    const T c = T(0.70710678118654752440084436210485);
    cplx<T> e[4] = {v[0], v[2], v[4], v[6]};
    cplx<T> o[4] = {v[1], v[3], v[5], v[7]};
    dft4<T, INV>(e);
    dft4<T, INV>(o);
    // o_k *= W8^k, W8 = exp(-+ 2 pi i / 8)
    cplx<T> o1 = o[1], o3 = o[3];
    if (!INV) {
        o[1] = mk<T>(c * (o1.x + o1.y), c * (o1.y - o1.x));
        o[3] = mk<T>(c * (o3.y - o3.x), -c * (o3.x + o3.y));
    } else {
        o[1] = mk<T>(c * (o1.x - o1.y), c * (o1.x + o1.y));
        o[3] = mk<T>(-c * (o3.x + o3.y), c * (o3.x - o3.y));
    }
    o[2] = mul_mj<cplx<T>, INV>(o[2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = cadd(e[k], o[k]);
        v[k + 4] = csub(e[k], o[k]);
    }
}

template <typename T, int R, bool INV> __device__ __forceinline__ void dftR(cplx<T>* v) {
    if (R == 2) dft2<T, INV>(v);
    else if (R == 4) dft4<T, INV>(v);
    else dft8<T, INV>(v);
}

// One Stockham stage of radix R at sub-transform size Ns, then recurse.
// PIN: the transform's input is zero in rows >= L/2 (the padding), so the
// first stage reads and transforms only its first R/2 inputs.  POUT: only
// rows < L/2 of the result are kept, so the last stage computes and stores
// only its first R/2 outputs.  Twiddles: W^r for r = 1, 2, 4 come from the
// table, the others are products of those.
template <typename T, int R, bool INV>
__device__ __forceinline__ void twiddle(cplx<T>* v, const cplx<T>* __restrict__ tw, int base) {
    auto cj = [](cplx<T> x) {
        if (INV) x.y = -x.y;
        return x;
    };
    const cplx<T> w1 = cj(tw[base]);
    v[1] = cmul(v[1], w1);
    if constexpr (R >= 4) {
        const cplx<T> w2 = cj(tw[2 * base]);
        const cplx<T> w3 = cmul(w1, w2);
        v[2] = cmul(v[2], w2);
        v[3] = cmul(v[3], w3);
        if constexpr (R >= 8) {
            const cplx<T> w4 = cj(tw[4 * base]);
            v[4] = cmul(v[4], w4);
            v[5] = cmul(v[5], cmul(w1, w4));
            v[6] = cmul(v[6], cmul(w2, w4));
            v[7] = cmul(v[7], cmul(w3, w4));
        }
    }
}

template <typename T, int L, int B, int NBS, int Ns, bool INV, bool PIN = false, bool POUT = false>
__device__ __forceinline__ void fft_stages(cplx<T>* s, const cplx<T>* __restrict__ tw, int col, int bslot) {
    if constexpr (Ns < L) {
        constexpr int REM = L / Ns;
        constexpr int R = REM >= 8 ? 8 : REM;
        constexpr int NBF = L / R;          // butterflies per column
        constexpr int PER = NBF / NBS;      // butterflies per thread
        static_assert(PER >= 1 && PER * NBS == NBF, "butterfly split");
        constexpr int LD = B + 1;
        constexpr bool FIRST_HALF = PIN && Ns == 1 && R >= 2;     // inputs r >= R/2 are zero
        constexpr bool LAST_HALF = POUT && Ns * R == L && R >= 2;  // outputs r >= R/2 unused
        constexpr int RIN = FIRST_HALF ? R / 2 : R, ROUT = LAST_HALF ? R / 2 : R;
        cplx<T> v[PER][R];
#pragma unroll
        for (int b = 0; b < PER; ++b) {
            const int j = bslot + b * NBS;
#pragma unroll
            for (int r = 0; r < R; ++r)
                v[b][r] = r < RIN ? s[(j + r * NBF) * LD + col] : mk<T>(T(0), T(0));
            if constexpr (Ns > 1) twiddle<T, R, INV>(v[b], tw, (j % Ns) * (LMAX / (Ns * R)));
            dftR<T, R, INV>(v[b]);
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < PER; ++b) {
            const int j = bslot + b * NBS;
            const int idx = (j / Ns) * Ns * R + (j % Ns);
#pragma unroll
            for (int r = 0; r < ROUT; ++r) s[(idx + r * Ns) * LD + col] = v[b][r];
        }
        __syncthreads();
        fft_stages<T, L, B, NBS, Ns * R, INV, false, POUT>(s, tw, col, bslot);
    }
}

// A full transform with the pruning flags chosen at run time.
template <typename T, int L, int B, int NBS, bool INV>
__device__ __forceinline__ void fft_run(cplx<T>* s, const cplx<T>* __restrict__ tw, int col, int bslot, bool pin,
                                        bool pout) {
    if (pin && pout) fft_stages<T, L, B, NBS, 1, INV, true, true>(s, tw, col, bslot);
    else if (pin) fft_stages<T, L, B, NBS, 1, INV, true, false>(s, tw, col, bslot);
    else if (pout) fft_stages<T, L, B, NBS, 1, INV, false, true>(s, tw, col, bslot);
    else fft_stages<T, L, B, NBS, 1, INV, false, false>(s, tw, col, bslot);
}

struct PassArgs {
    int n_in;        // rows loaded (rows n_in..L-1 are zero)
    int n_keep;      // rows stored
    int width;       // number of columns (strided pass) / lines (contiguous pass)
    long long in_row, out_row;       // stride between FFT rows (strided) / between lines (contig)
    long long in_plane, out_plane;   // stride between planes (strided pass)
    long long spec_row, spec_plane;  // spectrum strides (z pass)
    int spec_fold;                   // z pass: bit 0/1/2 = stored spectrum folded along columns/planes/rows
    int Lc, Lp;                      // z pass: full lengths along columns and planes (for the folding)
    int ngroups;     // column groups per plane
    int mode;        // 0 forward, 1 inverse, 2 forward*spec*inverse, 3 forward*conj(spec)*inverse
};

// FFT along a strided axis: CTA = (plane, group of B consecutive columns).
// Every thread issues its global loads in groups (up to 8) before it stores
// them to shared memory, so that their latencies overlap instead of forming
// a chain.
template <typename T, int L, int B, int NBS, bool Z>
__global__ void __launch_bounds__(B* NBS, sizeof(T) == 4 ? (B* NBS >= 512 ? 2 : (B* NBS >= 256 ? 3 : 1)) : 1) fft_strided_kernel(const cplx<T>* in, cplx<T>* out,
                                                              PassArgs a, const cplx<T>* __restrict__ tw,
                                                              const cplx<T>* __restrict__ spec) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
    constexpr int LD = B + 1;
    constexpr int NT = B * NBS;
    constexpr int EPT = L * B / NT;  // elements per thread
    const int plane = blockIdx.x / a.ngroups;
    const int c0 = (blockIdx.x % a.ngroups) * B;
    const int tid = threadIdx.x;
    const int col = tid % B, bslot = tid / B;
    const cplx<T> zero = mk<T>(T(0), T(0));
    const cplx<T>* ib = in + plane * a.in_plane + c0;
    const bool cok = c0 + col < a.width;   // i % B == col for every i = tid + k NT
    // loads in groups of at most 8 per thread, all of a group issued before
    // its shared-memory stores; the z pass also prefetches its spectrum
    // tile into registers when a thread holds at most 8 elements
    constexpr int G = EPT < 8 ? EPT : 8;
    constexpr bool PREF = EPT <= 8;
#pragma unroll
    for (int k0 = 0; k0 < EPT; k0 += G) {
        cplx<T> v[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int r = (tid + (k0 + g) * NT) / B;
            v[g] = (r < a.n_in && cok) ? ib[(long long)r * a.in_row + col] : zero;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) s[((tid + (k0 + g) * NT) / B) * LD + col] = v[g];
    }
    // spectrum element of (row r, this plane, this column), folded along the
    // axes where only frequencies 0..L/2 are stored
    const int xc = c0 + col, pl = plane;
    const int fxc = (a.spec_fold & 1) ? min(xc, a.Lc - xc) : xc;
    const int fpl = (a.spec_fold & 2) ? min(pl, a.Lp - pl) : pl;
    const cplx<T>* spb = spec + fpl * a.spec_plane + fxc;
    auto srow = [&](int r) { return (long long)((a.spec_fold & 4) ? min(r, L - r) : r) * a.spec_row; };
    cplx<T> sp[PREF && Z ? EPT : 1];
    if constexpr (PREF && Z) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int r = (tid + k * NT) / B;
            sp[k] = cok ? spb[srow(r)] : zero;
        }
    }
    __syncthreads();
    const bool half_in = 2 * a.n_in <= L, half_out = 2 * a.n_keep <= L;
    if (!Z && a.mode == 1) {
        fft_run<T, L, B, NBS, true>(s, tw, col, bslot, false, half_out);
    } else {
        // forward: the z pass keeps the whole spectrum for the product
        fft_run<T, L, B, NBS, false>(s, tw, col, bslot, half_in, !Z && half_out);
    }
    if constexpr (Z) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int r = (tid + k * NT) / B;
            cplx<T> w;
            if constexpr (PREF && Z) w = sp[k];
            else w = cok ? spb[srow(r)] : zero;
            if (a.mode == 3) w.y = -w.y;
            s[r * LD + col] = cmul(s[r * LD + col], w);
        }
        __syncthreads();
        fft_run<T, L, B, NBS, true>(s, tw, col, bslot, false, half_out);
    }
    cplx<T>* ob = out + plane * a.out_plane + c0;
    if (cok) {
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
            const int r = (tid + k * NT) / B;
            if (r < a.n_keep) ob[r * a.out_row + col] = s[r * LD + col];
        }
    }
}

// FFT along contiguous lines: CTA = B consecutive lines, transposed in smem.
template <typename T, int L, int B, int NBS>
__global__ void __launch_bounds__(B* NBS) fft_contig_kernel(const cplx<T>* in, cplx<T>* out,
                                                             PassArgs a, const cplx<T>* __restrict__ tw) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cplx<T>* s = reinterpret_cast<cplx<T>*>(smem_raw);
    constexpr int LD = B + 1;
    constexpr int NT = B * NBS;
    constexpr int EPT = L * B / NT;
    const int l0 = blockIdx.x * B;
    const int tid = threadIdx.x;
    const int col = tid % B, bslot = tid / B;
    const cplx<T> zero = mk<T>(T(0), T(0));
    cplx<T> v[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int i = tid + k * NT;
        const int c = i / L, x = i % L;
        v[k] = (x < a.n_in && l0 + c < a.width) ? in[(long long)(l0 + c) * a.in_row + x] : zero;
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int i = tid + k * NT;
        s[(i % L) * LD + i / L] = v[k];
    }
    __syncthreads();
    const bool half_in = 2 * a.n_in <= L, half_out = 2 * a.n_keep <= L;
    if (a.mode == 1) fft_run<T, L, B, NBS, true>(s, tw, col, bslot, false, half_out);
    else fft_run<T, L, B, NBS, false>(s, tw, col, bslot, half_in, half_out);
    for (int i = tid; i < a.n_keep * B; i += NT) {
        const int c = i / a.n_keep, x = i % a.n_keep;
        if (l0 + c < a.width) out[(long long)(l0 + c) * a.out_row + x] = s[x * LD + c];
    }
}

template <typename T> struct TileCfg;
// columns per CTA by length: one 128-byte line per row at most, and a few
// elements per thread, so that several CTAs fit on an SM.
template <> struct TileCfg<float> {
    static constexpr int B(int L) { return L <= 64 ? 32 : (L <= 512 ? 16 : 8); }
};
template <> struct TileCfg<double> {
    static constexpr int B(int L) { return L <= 128 ? 16 : (L == 256 ? 8 : 4); }
};
// strided passes: narrower column groups at the long lengths, so that a
// thread holds at most 8 elements (registers) and two CTAs fit on an SM
template <typename T> struct TileCfgS;
template <> struct TileCfgS<float> {
    static constexpr int B(int L) { return L <= 64 ? 32 : (L <= 512 ? 16 : 8); }
};
template <> struct TileCfgS<double> {
    static constexpr int B(int L) { return L <= 128 ? 16 : (L == 256 ? 8 : 4); }
};

template <typename T, int L>
pim_status launch_len(const cplx<T>* in, cplx<T>* out, PassArgs a, const cplx<T>* tw, cudaStream_t s) {
    constexpr int B = TileCfg<T>::B(L);
    constexpr int NBS0 = L / 8 > 0 ? L / 8 : 1;
    constexpr int NBS = NBS0 * B > 512 ? 512 / B : NBS0;
    constexpr int NT = B * NBS;
    const size_t smem = (size_t)L * (B + 1) * sizeof(cplx<T>);
    auto k = fft_contig_kernel<T, L, B, NBS>;
    PIM_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int grid = (a.width + B - 1) / B;
    if (grid > 0) k<<<grid, NT, smem, s>>>(in, out, a, tw);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <typename T, int L>
pim_status launch_strided_len(const cplx<T>* in, cplx<T>* out, PassArgs a, int nplanes, const cplx<T>* tw,
                              const cplx<T>* spec, cudaStream_t s) {
    constexpr int B = TileCfgS<T>::B(L);
    constexpr int NBS0 = L / 8 > 0 ? L / 8 : 1;
    constexpr int NBS = NBS0 * B > 512 ? 512 / B : NBS0;
    constexpr int NT = B * NBS;
    const size_t smem = (size_t)L * (B + 1) * sizeof(cplx<T>);
    auto k = a.mode >= 2 ? fft_strided_kernel<T, L, B, NBS, true> : fft_strided_kernel<T, L, B, NBS, false>;
    PIM_CK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    a.ngroups = (a.width + B - 1) / B;
    const long long grid = (long long)a.ngroups * nplanes;
    if (grid > 0) k<<<(unsigned)grid, NT, smem, s>>>(in, out, a, tw, spec);
    PIM_CK(cudaGetLastError());
    return PIM_OK;
}

template <typename T>
pim_status pass_contig(int L, const cplx<T>* in, cplx<T>* out, PassArgs a, const cplx<T>* tw, cudaStream_t s) {
    switch (L) {
        case 16: return launch_len<T, 16>(in, out, a, tw, s);
        case 32: return launch_len<T, 32>(in, out, a, tw, s);
        case 64: return launch_len<T, 64>(in, out, a, tw, s);
        case 128: return launch_len<T, 128>(in, out, a, tw, s);
        case 256: return launch_len<T, 256>(in, out, a, tw, s);
        case 512: return launch_len<T, 512>(in, out, a, tw, s);
        case 1024: return launch_len<T, 1024>(in, out, a, tw, s);
        default: pim_set_error("FFT length not supported"); return PIM_ERR_UNSUPPORTED;
    }
}

template <typename T>
pim_status pass_strided(int L, const cplx<T>* in, cplx<T>* out, PassArgs a, int nplanes, const cplx<T>* tw,
                        const cplx<T>* spec, cudaStream_t s) {
    switch (L) {
        case 16: return launch_strided_len<T, 16>(in, out, a, nplanes, tw, spec, s);
        case 32: return launch_strided_len<T, 32>(in, out, a, nplanes, tw, spec, s);
        case 64: return launch_strided_len<T, 64>(in, out, a, nplanes, tw, spec, s);
        case 128: return launch_strided_len<T, 128>(in, out, a, nplanes, tw, spec, s);
        case 256: return launch_strided_len<T, 256>(in, out, a, nplanes, tw, spec, s);
        case 512: return launch_strided_len<T, 512>(in, out, a, nplanes, tw, spec, s);
        case 1024: return launch_strided_len<T, 1024>(in, out, a, nplanes, tw, spec, s);
        default: pim_set_error("FFT length not supported"); return PIM_ERR_UNSUPPORTED;
    }
}

template <typename T> const cplx<T>* twiddles(pim_plan P);
template <> const float2* twiddles<float>(pim_plan P) { return P->tw32; }
template <> const double2* twiddles<double>(pim_plan P) { return P->tw64; }

}  // namespace

pim_status fft_make_twiddles(pim_plan P) {
    std::vector<float2> t32(LMAX);
    std::vector<double2> t64(LMAX);
    for (int j = 0; j < LMAX; ++j) {
        // exp(-2 pi i j / LMAX), angles reduced to the first octant by symmetry
        // are not needed: long double evaluation rounded once.
        long double th = -2.0L * 3.141592653589793238462643383279502884L * (long double)j / (long double)LMAX;
        double c = (double)cosl(th), s = (double)sinl(th);
        t64[j] = make_double2(c, s);
        t32[j] = make_float2((float)cosl(th), (float)sinl(th));
    }
    pim_status st;
    if ((st = pim_alloc(P, (void**)&P->tw32, LMAX * sizeof(float2))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&P->tw64, LMAX * sizeof(double2))) != PIM_OK) return st;
    PIM_CK(cudaMemcpy(P->tw32, t32.data(), LMAX * sizeof(float2), cudaMemcpyHostToDevice));
    PIM_CK(cudaMemcpy(P->tw64, t64.data(), LMAX * sizeof(double2), cudaMemcpyHostToDevice));
    return PIM_OK;
}

// Pruned 3D convolution U = IFFT(FFT(pad(A)) .* spec) restricted to the data
// nodes.  A [nz][ny][nx] in, result written back to A.  B [nz][ny][Lx] and
// C [nz][Ly][Lx] are work buffers; spec is [Lz][Ly][Lx] (already scaled by
// 1 / (Lx Ly Lz)).  conj_spec selects the adjoint (conjugated spectrum).
template <typename T>
pim_status fft3_conv(pim_plan P, const FftGeom& g, cplx<T>* A, cplx<T>* B, cplx<T>* C, const cplx<T>* spec,
                     bool conj_spec, cudaStream_t s) {
    const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
    const cplx<T>* tw = twiddles<T>(P);
    pim_status st;
    PassArgs a{};
    // x forward: nz*ny lines of nx -> Lx
    a = PassArgs{};
    a.n_in = nx; a.n_keep = Lx; a.width = nz * ny; a.in_row = nx; a.out_row = Lx; a.mode = 0;
    if ((st = pass_contig<T>(Lx, A, B, a, tw, s)) != PIM_OK) return st;
    // y forward: planes z, rows y (stride Lx), columns x' (Lx)
    a = PassArgs{};
    a.n_in = ny; a.n_keep = Ly; a.width = Lx; a.in_row = Lx; a.out_row = Lx;
    a.in_plane = (long long)ny * Lx; a.out_plane = (long long)Ly * Lx; a.mode = 0;
    if ((st = pass_strided<T>(Ly, B, C, a, nz, tw, nullptr, s)) != PIM_OK) return st;
    // z forward * spectrum * inverse: planes y' (stride Lx), rows z (stride Ly Lx)
    a = PassArgs{};
    a.n_in = nz; a.n_keep = nz; a.width = Lx; a.in_row = (long long)Ly * Lx; a.out_row = (long long)Ly * Lx;
    a.in_plane = Lx; a.out_plane = Lx;
    if (g.fold || g.S[0]) {
        a.spec_row = (long long)g.S[1] * g.S[0]; a.spec_plane = g.S[0];
        a.spec_fold = g.fold; a.Lc = Lx; a.Lp = Ly;
    } else {
        a.spec_row = (long long)Ly * Lx; a.spec_plane = Lx;
    }
    a.mode = conj_spec ? 3 : 2;
    if ((st = pass_strided<T>(Lz, C, C, a, Ly, tw, spec, s)) != PIM_OK) return st;
    // y inverse: keep ny rows
    a = PassArgs{};
    a.n_in = Ly; a.n_keep = ny; a.width = Lx; a.in_row = Lx; a.out_row = Lx;
    a.in_plane = (long long)Ly * Lx; a.out_plane = (long long)ny * Lx; a.mode = 1;
    if ((st = pass_strided<T>(Ly, C, B, a, nz, tw, nullptr, s)) != PIM_OK) return st;
    // x inverse: keep nx
    a = PassArgs{};
    a.n_in = Lx; a.n_keep = nx; a.width = nz * ny; a.in_row = Lx; a.out_row = nx; a.mode = 1;
    return pass_contig<T>(Lx, B, A, a, tw, s);
}

// Full forward 3D FFT of X [Lz][Ly][Lx] in place (tables at plan time).
template <typename T>
pim_status fft3_forward_full(pim_plan P, const FftGeom& g, cplx<T>* X, cplx<T>* tmp, cudaStream_t s) {
    (void)tmp;
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2];
    const cplx<T>* tw = twiddles<T>(P);
    pim_status st;
    PassArgs a{};
    a.n_in = Lx; a.n_keep = Lx; a.width = Lz * Ly; a.in_row = Lx; a.out_row = Lx; a.mode = 0;
    if ((st = pass_contig<T>(Lx, X, X, a, tw, s)) != PIM_OK) return st;
    a = PassArgs{};
    a.n_in = Ly; a.n_keep = Ly; a.width = Lx; a.in_row = Lx; a.out_row = Lx;
    a.in_plane = (long long)Ly * Lx; a.out_plane = (long long)Ly * Lx; a.mode = 0;
    if ((st = pass_strided<T>(Ly, X, X, a, Lz, tw, nullptr, s)) != PIM_OK) return st;
    a = PassArgs{};
    a.n_in = Lz; a.n_keep = Lz; a.width = Lx; a.in_row = (long long)Ly * Lx; a.out_row = (long long)Ly * Lx;
    a.in_plane = Lx; a.out_plane = Lx; a.mode = 0;
    return pass_strided<T>(Lz, X, X, a, Ly, tw, nullptr, s);
}

template pim_status fft3_conv<float>(pim_plan, const FftGeom&, float2*, float2*, float2*, const float2*, bool,
                                     cudaStream_t);
template pim_status fft3_conv<double>(pim_plan, const FftGeom&, double2*, double2*, double2*, const double2*, bool,
                                      cudaStream_t);
template pim_status fft3_forward_full<float>(pim_plan, const FftGeom&, float2*, float2*, cudaStream_t);
template pim_status fft3_forward_full<double>(pim_plan, const FftGeom&, double2*, double2*, cudaStream_t);
