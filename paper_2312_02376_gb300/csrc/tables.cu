// Plan-time tables: the near-zone kernel spectrum (Sec. 3.3 step 2) and the
// far-zone table G_far = G^p - G_near on the shifted far grids (Sec. 3.2).
// Everything here is FP64.
#include <cmath>
#include <complex>
#include <vector>

#include "pim_internal.cuh"

namespace {

constexpr double PI = 3.141592653589793238462643383279502884;
constexpr double EULER_GAMMA = 0.57721566490153286060651209008240243;

// exp(-j k R) / (4 pi R), k = k + j ki (ki <= 0: a lossy medium)
__device__ __forceinline__ double2 G0(double R, double k, double ki) {
    double s, c;
    sincos(k * R, &s, &c);
    double a = 1.0 / (4.0 * PI * R);
    if (ki != 0.0) a *= exp(ki * R);
    return make_double2(c * a, -s * a);
}

// ---------------------------------------------------------------------------
// near-zone kernel on the padded grid
// K(delta) = sum_i exp(-j k0.(i o L)) g(delta - i o (n-1)), g(e) = G0(|e o h|),
// g(0) = 0, for delta in [-(n-1), n-1]^3 placed circularly (index delta mod L)
// ---------------------------------------------------------------------------
struct NearArgs {
    int n[3], L[3];
    double h[3], k, ki;
    int nimg;
    const int* img;          // nimg x 3
    const double2* phase;    // nimg
};

__global__ void near_table_kernel(NearArgs a, double2* out) {
    const long long total = (long long)a.L[0] * a.L[1] * a.L[2];
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int idx[3] = {(int)(e % a.L[0]), (int)((e / a.L[0]) % a.L[1]), (int)(e / ((long long)a.L[0] * a.L[1]))};
        int dl[3];
        bool used = true;
        for (int d = 0; d < 3; ++d) {
            if (idx[d] <= a.n[d] - 1) dl[d] = idx[d];
            else if (idx[d] >= a.L[d] - (a.n[d] - 1)) dl[d] = idx[d] - a.L[d];
            else used = false;
        }
        double2 acc = make_double2(0.0, 0.0);
        if (used) {
            for (int i = 0; i < a.nimg; ++i) {
                double r2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double x = (double)(dl[d] - a.img[3 * i + d] * (a.n[d] - 1)) * a.h[d];
                    r2 += x * x;
                }
                if (r2 == 0.0) continue;  // g(0) = 0
                acc = cadd(acc, cmul(a.phase[i], G0(sqrt(r2), a.k, a.ki)));
            }
        }
        out[e] = acc;
    }
}

template <typename T>
__global__ void scale_convert_kernel(const double2* in, cplx<T>* out, long long n, double s) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        out[i] = mk<T>((T)(in[i].x * s), (T)(in[i].y * s));
    }
}

// the kept part [Sz][Sy][Sx] of a full spectrum [Lz][Ly][Lx], scaled
template <typename T>
__global__ void fold_convert_kernel(const double2* in, cplx<T>* out, int Lx, int Ly, int Sx, int Sy, int Sz, double s) {
    const long long tot = (long long)Sx * Sy * Sz;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Sx), y = (int)((i / Sx) % Sy), z = (int)(i / ((long long)Sx * Sy));
        const double2 v = in[((long long)z * Ly + y) * Lx + x];
        out[i] = mk<T>((T)(v.x * s), (T)(v.y * s));
    }
}

// ---------------------------------------------------------------------------
// special functions (FP64)
// ---------------------------------------------------------------------------
// K0(x), x > 0.  x <= 2: the power series
//   K0(x) = -(ln(x/2) + gamma) I0(x) + sum_{k>=1} (x^2/4)^k / (k!)^2 H_k
// (Abramowitz & Stegun 9.6.13 with 9.6.12); x > 2: the trapezoidal rule with
// step 0.1 on K0(x) = int_0^inf exp(-x cosh t) dt, which converges
// exponentially for this analytic integrand (Trefethen & Weideman, SIAM Rev.
// 56 (2014)).  Relative error below 1e-14 over (0, inf).
__device__ double bessel_k0(double x) {
    if (x <= 2.0) {
        const double y = 0.25 * x * x;
        double t = 1.0, I = 1.0, S = 0.0, H = 0.0;
        for (int k = 1; k < 40; ++k) {
            t *= y / ((double)k * (double)k);
            H += 1.0 / k;
            I += t;
            S += t * H;
            if (t < 1e-18 * I) break;
        }
        return -(log(0.5 * x) + EULER_GAMMA) * I + S;
    }
    const double h = 0.1;
    double s = 0.5 * exp(-x);
    for (int k = 1; k < 400; ++k) {
        const double c = cosh(k * h);
        s += exp(-x * c);
        if (x * (c - 1.0) > 42.0) break;
    }
    return h * s;
}

// ---------------------------------------------------------------------------
// far-zone table, one CTA per entry
// ---------------------------------------------------------------------------
struct FarArgs {
    int nf[3];
    double df[3];
    int perm[3];         // canonical axis order: periodic axes first
    int npd;
    double Lc[3];        // canonical periods (free axes: unused)
    double k;
    double k0c[3];       // canonical phase shifts
    int npsp;
    double D[3];
    int nimg;
    const int* img;
    const double2* phase;
    // 3D lattice, Eq. pgf_3: bit c set when axis c may serve as the series'
    // image axis (no Floquet mode of the other two axes has k_z = 0); each
    // entry takes the allowed axis along which its terms decay fastest
    int zaxes;
    // complex k (ki) or phase shift (k0ci): the series in complex arithmetic
    int cplx;
    double ki;
    double k0ci[3];
    int* bad;            // set when a Hankel-function argument is outside the evaluated regimes
};

constexpr int FAR_NT = 128;

__device__ __forceinline__ double2 cexpj(double th) {  // exp(j th)
    double s, c;
    sincos(th, &s, &c);
    return make_double2(c, s);
}

// exp(-j z t) for complex z
__device__ __forceinline__ double2 cexp_mj(double2 z, double t) {
    // -j (zr + j zi) t = zi t - j zr t
    const double m = exp(z.y * t);
    double s, c;
    sincos(z.x * t, &s, &c);
    return make_double2(m * c, -m * s);
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// kz = sqrt(r) with Im <= 0 for real r (positive root for r > 0)
__device__ __forceinline__ double2 kz_branch(double r) {
    return r >= 0.0 ? make_double2(sqrt(r), 0.0) : make_double2(0.0, -sqrt(-r));
}

// principal square root, then the branch with Im <= 0 (Sec. 2 after Eq. pgf;
// for a positive real radicand the positive root)
__device__ __forceinline__ double2 csqrt_branch(double2 w) {
    const double r = hypot(w.x, w.y);
    if (r == 0.0) return make_double2(0.0, 0.0);
    const double t = sqrt(0.5 * (r + fabs(w.x)));
    double2 v = w.x >= 0.0 ? make_double2(t, w.y / (2.0 * t)) : make_double2(fabs(w.y) / (2.0 * t), copysign(t, w.y));
    if (v.y > 0.0) v = make_double2(-v.x, -v.y);
    return v;
}

__device__ __forceinline__ double2 cexp_c(double2 z) {  // exp(z)
    const double m = exp(z.x);
    double s, c;
    sincos(z.y, &s, &c);
    return make_double2(m * c, m * s);
}

// K0(w) for complex w with Re w >= 0, w != 0 (the 1D series with complex k
// or k0: H0^(2)(z) = (2j/pi) K0(j z)).  Three methods, each within about
// 1e-13 relative where it is used (checked against an independent library
// on a grid of |w| <= 40, |arg w| <= pi/2):
//  |w| >= 20: the asymptotic series sqrt(pi/2w) e^-w sum_k c_k w^-k,
//    c_k = c_{k-1} (-(2k-1)^2) / (8k) (A&S 9.7.2), summed to its smallest term;
//  |w| <= 2, and |w| <= 6 within 0.17 rad of the imaginary axis: the power
//    series of A&S 9.6.13 with 9.6.12 (complex logarithm); near the real axis
//    K0 ~ e^-|w| while the terms grow like e^|w|, so it is not used there;
//  |arg w| <= 1.4: the trapezoidal rule on K0(w) = int_0^inf exp(-w cosh t) dt,
//    whose integrand is analytic and decaying in the strip |Im t| < d,
//    d = pi/2 - |arg w| (Trefethen & Weideman, SIAM Rev. 56 (2014)): on the
//    line Im t = s = d/2 it is at most exp(-|w| cos(|arg w| + s)), so the step
//    h = 2 pi s / (42 + |w| (cos|arg w| - cos(|arg w| + s))) keeps the error
//    below e^-42 relative to K0 ~ exp(-|w| cos arg w).
// Other arguments (modulus 6..20 within 0.17 rad of the imaginary axis:
// weakly lossy propagating modes far from the axis) set *bad and return 0.
__device__ double2 bessel_k0c(double2 w, int* bad) {
    const double aw = hypot(w.x, w.y), th = atan2(w.y, w.x);
    if (aw >= 20.0) {
        const double2 iw = cdiv(make_double2(1.0, 0.0), w);
        double2 term = make_double2(1.0, 0.0), sum = term;
        double last = 1.0;
        for (int k = 1; k < 60; ++k) {
            const double f = -(2.0 * k - 1.0) * (2.0 * k - 1.0) / (8.0 * k);
            term = cmul(term, iw);
            term.x *= f;
            term.y *= f;
            const double mt = hypot(term.x, term.y);
            if (mt > last) break;  // the smallest term has been passed
            sum = cadd(sum, term);
            last = mt;
            if (mt < 1e-17) break;
        }
        const double2 pre = csqrt_branch(cdiv(make_double2(0.5 * PI, 0.0), w));
        // the principal root (Re w >= 0): undo the Im <= 0 choice when it flipped
        const double2 root = pre.x < 0.0 ? make_double2(-pre.x, -pre.y) : pre;
        return cmul(cmul(root, cexp_c(make_double2(-w.x, -w.y))), sum);
    }
    if (aw <= 2.0 || (aw <= 6.0 && fabs(th) > 1.4)) {
        const double2 y = make_double2(0.25 * (w.x * w.x - w.y * w.y), 0.5 * w.x * w.y);
        double2 t = make_double2(1.0, 0.0), I = t, S = make_double2(0.0, 0.0);
        double H = 0.0;
        for (int k = 1; k < 80; ++k) {
            t = cmul(t, y);
            t.x /= (double)k * (double)k;
            t.y /= (double)k * (double)k;
            H += 1.0 / k;
            I = cadd(I, t);
            S = cadd(S, make_double2(t.x * H, t.y * H));
            if (k > 8 && hypot(t.x, t.y) < 1e-18 * hypot(I.x, I.y)) break;
        }
        const double2 lg = make_double2(log(0.5 * aw) + EULER_GAMMA, th);  // log(w/2) + gamma
        return csub(S, cmul(lg, I));
    }
    if (fabs(th) <= 1.4) {
        const double at = fabs(th), sd = 0.5 * (0.5 * PI - at);
        const double h = fmin(0.1, 2.0 * PI * sd / (42.0 + aw * (cos(at) - cos(at + sd))));
        double2 sum = cexp_c(make_double2(-w.x, -w.y));
        sum.x *= 0.5;
        sum.y *= 0.5;
        for (int k = 1; k < 20000; ++k) {
            const double c = cosh(k * h);
            sum = cadd(sum, cexp_c(make_double2(-w.x * c, -w.y * c)));
            if (w.x * (c - 1.0) > 44.0) break;
        }
        return make_double2(h * sum.x, h * sum.y);
    }
    atomicOr(bad, 1);
    return make_double2(0.0, 0.0);
}

__device__ int mode_window(double kc, double Lc, double decay_len, double k) {
    const double kmax = 42.0 / decay_len + fabs(k) + fabs(kc);
    return (int)ceil(kmax * Lc / (2.0 * PI)) + 4;
}

__global__ void __launch_bounds__(FAR_NT) far_table_kernel(FarArgs a, double2* out) {
    __shared__ double2 red[FAR_NT];
    const int e = blockIdx.x;
    const int W0 = 2 * a.nf[0] - 1, W1 = 2 * a.nf[1] - 1;
    const int idx[3] = {e % W0, (e / W0) % W1, e / (W0 * W1)};
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = (double)(idx[d] - (a.nf[d] - 1)) * a.df[d] + 0.5 * a.df[d];
    const double x = r[a.perm[0]], y = r[a.perm[1]], z = r[a.perm[2]];
    const double Lx = a.Lc[0], Ly = a.Lc[1], Lz = a.Lc[2];
    const int tid = threadIdx.x;
    double2 acc = make_double2(0.0, 0.0);
    double2 fixed = make_double2(0.0, 0.0);  // terms added once (by thread 0)

    if (a.npsp) {
        // ------------------------- Eq. lgf ---------------------------------
        // (1/(pi Lx)) sum_{m>=1} sum_{lattice rho} K0(2 pi m rho / Lx) cos(2 pi m x / Lx)
        const double rmax = 42.0 * Lx / (2.0 * PI) + (a.npd >= 2 ? Ly : 0.0) + (a.npd >= 3 ? Lz : 0.0);
        const int NN = a.npd >= 2 ? (int)ceil(rmax / Ly) + 1 : 0;
        const int KK = a.npd >= 3 ? (int)ceil(rmax / Lz) + 1 : 0;
        const int npairs = (2 * NN + 1) * (2 * KK + 1);
        for (int t = tid; t < npairs; t += FAR_NT) {
            const int nn = t % (2 * NN + 1) - NN, kk = t / (2 * NN + 1) - KK;
            double rho;
            if (a.npd == 1) rho = hypot(y, z);
            else if (a.npd == 2) rho = hypot(nn * Ly + y, z);
            else rho = hypot(nn * Ly + y, kk * Lz + z);
            if (a.npd >= 2 && rho > rmax) continue;
            const int mmax = (int)ceil(42.0 * Lx / (2.0 * PI * rho)) + 2;
            double s = 0.0;
            for (int m = mmax; m >= 1; --m)
                s += bessel_k0(2.0 * PI * m * rho / Lx) * cos(2.0 * PI * m * x / Lx);
            acc.x += s / (PI * Lx);
        }
        if (a.npd == 3) {
            const int K = (int)ceil(42.0 * Ly / (2.0 * PI * Lz)) + 2;
            for (int kk = -K + tid; kk <= K; kk += FAR_NT) {
                const double aa = exp(-2.0 * PI * fabs(kk * Lz + z) / Ly);
                acc.x -= log1p(-2.0 * aa * cos(2.0 * PI * y / Ly) + aa * aa) / (4.0 * PI * Lx);
            }
            if (tid == 0) fixed.x = (z * z - fabs(z) * Lz) / (2.0 * Lx * Ly * Lz);
        } else if (a.npd == 2) {
            if (tid == 0) {
                const double aa = exp(-2.0 * PI * fabs(z) / Ly);
                fixed.x = -fabs(z) / (2.0 * Lx * Ly) - log1p(-2.0 * aa * cos(2.0 * PI * y / Ly) + aa * aa) / (4.0 * PI * Lx);
            }
        } else {
            if (tid == 0) fixed.x = -log(hypot(y, z)) / (2.0 * PI * Lx);
        }
    } else if (a.npd == 1 && a.cplx) {
        // ---------------- Eq. pgf_1, complex k or k0 -----------------------
        // exp(-j kx x) H0^(2)(krho rho) / (4 j Lx) = exp(-j kx x) K0(j krho rho) / (2 pi Lx)
        const double rho = hypot(y, z);
        const int M = mode_window(hypot(a.k0c[0], a.k0ci[0]), Lx, rho, hypot(a.k, a.ki));
        const double2 kk = make_double2(a.k * a.k - a.ki * a.ki, 2.0 * a.k * a.ki);
        for (int t = tid; t < 2 * M + 1; t += FAR_NT) {
            const int m = t - M;
            const double2 kx = make_double2(a.k0c[0] + 2.0 * PI * m / Lx, a.k0ci[0]);
            const double2 krho = csqrt_branch(csub(kk, cmul(kx, kx)));
            const double2 w = make_double2(-krho.y * rho, krho.x * rho);  // j krho rho
            const double2 k0v = bessel_k0c(w, a.bad);
            const double2 h = make_double2(k0v.x / (2.0 * PI * Lx), k0v.y / (2.0 * PI * Lx));
            acc = cadd(acc, cmul(cexp_mj(kx, x), h));
        }
    } else if (a.npd == 1) {
        // ------------------------- Eq. pgf_1 -------------------------------
        const double rho = hypot(y, z);
        const int M = mode_window(a.k0c[0], Lx, rho, a.k);
        for (int t = tid; t < 2 * M + 1; t += FAR_NT) {
            const int m = t - M;
            const double kx = a.k0c[0] + 2.0 * PI * m / Lx;
            const double rad = a.k * a.k - kx * kx;
            double2 h;  // H0^(2)(krho rho) / (4 j Lx)
            if (rad > 0.0) {
                const double arg = sqrt(rad) * rho;
                // (J0 - j Y0) / (4 j Lx) = (-Y0 - j J0) / (4 Lx)
                h = make_double2(-y0(arg) / (4.0 * Lx), -j0(arg) / (4.0 * Lx));
            } else {
                // krho = -j kappa: H0^(2)(-j kappa rho) = (2j/pi) K0(kappa rho)
                h = make_double2(bessel_k0(sqrt(-rad) * rho) / (2.0 * PI * Lx), 0.0);
            }
            acc = cadd(acc, cmul(cexpj(-kx * x), h));
        }
    } else {
        // ------------------------- Eq. pgf_2 / pgf_3 -----------------------
        // For the 3D lattice the sum is the same whichever axis plays z: the
        // modes needed grow as Lx Ly / dlen^2 (dlen the distance to the
        // nearest image plane along z), so the axis with the largest
        // Lz dlen^2 is taken (among those allowed by a.zaxes).
        double xs = x, ys = y, zs = z, Lxs = Lx, Lys = Ly, Lzs = Lz;
        double k0x = a.k0c[0], k0y = a.k0c[1], k0z = a.k0c[2];
        double k0xi = a.k0ci[0], k0yi = a.k0ci[1], k0zi = a.k0ci[2];
        if (a.npd == 3) {
            int cz = 2;
            double best = -1.0;
            for (int c = 0; c < 3; ++c) {
                if (!(a.zaxes & (1 << c))) continue;
                const double dl = fmin(fabs(r[c]), a.Lc[c] - fabs(r[c]));
                const double score = a.Lc[c] * dl * dl;
                if (score > best) {
                    best = score;
                    cz = c;
                }
            }
            const int c1 = cz == 0 ? 1 : 0, c2 = cz == 2 ? 1 : 2;  // the other two, in order
            xs = r[c1];
            ys = r[c2];
            zs = r[cz];
            Lxs = a.Lc[c1];
            Lys = a.Lc[c2];
            Lzs = a.Lc[cz];
            k0x = a.k0c[c1];
            k0y = a.k0c[c2];
            k0z = a.k0c[cz];
            k0xi = a.k0ci[c1];
            k0yi = a.k0ci[c2];
            k0zi = a.k0ci[cz];
        }
        const double dlen = a.npd == 2 ? fabs(zs) : fmin(fabs(zs), Lzs - fabs(zs));
        const double kabs = a.cplx ? hypot(a.k, a.ki) : a.k;
        const int M = mode_window(a.cplx ? hypot(k0x, k0xi) : k0x, Lxs, dlen, kabs);
        const int N = mode_window(a.cplx ? hypot(k0y, k0yi) : k0y, Lys, dlen, kabs);
        const int W = 2 * N + 1;
        const long long nm = (long long)(2 * M + 1) * W;
        const double A = Lxs * Lys;
        if (a.cplx) {
            // the same series in complex arithmetic: kx, ky carry the phase
            // shift's imaginary parts, kz = (k^2 - kx^2 - ky^2)^(1/2) with Im <= 0
            const double2 kk = make_double2(a.k * a.k - a.ki * a.ki, 2.0 * a.k * a.ki);
            const double2 kz0 = make_double2(k0z, k0zi), mkz0 = make_double2(-k0z, -k0zi);
            const double2 one = make_double2(1.0, 0.0);
            for (long long t = tid; t < nm; t += FAR_NT) {
                const int m = (int)(t / W) - M, n = (int)(t % W) - N;
                const double2 kx = make_double2(k0x + 2.0 * PI * m / Lxs, k0xi);
                const double2 ky = make_double2(k0y + 2.0 * PI * n / Lys, k0yi);
                const double2 kz = csqrt_branch(csub(csub(kk, cmul(kx, kx)), cmul(ky, ky)));
                double2 zf = cexp_mj(kz, fabs(zs));
                if (a.npd == 3) {
                    const double2 em = cexp_mj(csub(kz, kz0), Lzs), ep = cexp_mj(cadd(kz, kz0), Lzs);
                    const double2 t2 = cdiv(cmul(cexp_mj(kz, Lzs + zs), cexp_mj(mkz0, Lzs)), csub(one, em));
                    const double2 t3 = cdiv(cmul(cexp_mj(kz, Lzs - zs), cexp_mj(kz0, Lzs)), csub(one, ep));
                    zf = cadd(zf, cadd(t2, t3));
                }
                const double2 den = make_double2(-2.0 * kz.y * A, 2.0 * kz.x * A);
                const double2 ph = cexp_mj(make_double2(kx.x * xs + ky.x * ys, kx.y * xs + ky.y * ys), 1.0);
                acc = cadd(acc, cmul(ph, cdiv(zf, den)));
            }
        } else
        for (long long t = tid; t < nm; t += FAR_NT) {
            const int m = (int)(t / W) - M, n = (int)(t % W) - N;
            const double kx = k0x + 2.0 * PI * m / Lxs;
            const double ky = k0y + 2.0 * PI * n / Lys;
            const double2 kz = kz_branch(a.k * a.k - kx * kx - ky * ky);
            double2 zf = cexp_mj(kz, fabs(zs));
            if (a.npd == 3) {
                // z-image factor of Eq. pgf_3; numerators with their exponents
                // combined: e^{-j kz (Lz + z)} e^{j kz0 Lz}, e^{-j kz (Lz - z)} e^{-j kz0 Lz}
                const double2 km = make_double2(kz.x - k0z, kz.y), kp = make_double2(kz.x + k0z, kz.y);
                const double2 em = cexp_mj(km, Lzs), ep = cexp_mj(kp, Lzs);
                const double2 one = make_double2(1.0, 0.0);
                const double2 t2 = cdiv(cmul(cexp_mj(kz, Lzs + zs), cexpj(k0z * Lzs)), csub(one, em));
                const double2 t3 = cdiv(cmul(cexp_mj(kz, Lzs - zs), cexpj(-k0z * Lzs)), csub(one, ep));
                zf = cadd(zf, cadd(t2, t3));
            }
            // / (2 j kz A)
            const double2 den = make_double2(-2.0 * kz.y * A, 2.0 * kz.x * A);
            acc = cadd(acc, cmul(cexpj(-(kx * xs + ky * ys)), cdiv(zf, den)));
        }
    }
    red[tid] = acc;
    __syncthreads();
    for (int st = FAR_NT / 2; st > 0; st >>= 1) {
        if (tid < st) red[tid] = cadd(red[tid], red[tid + st]);
        __syncthreads();
    }
    if (tid == 0) {
        double2 v = cadd(red[0], fixed);
        // subtract the near images (Eq. 4)
        for (int i = 0; i < a.nimg; ++i) {
            double r2 = 0.0;
            for (int d = 0; d < 3; ++d) {
                const double q = r[d] - a.img[3 * i + d] * a.D[d];
                r2 += q * q;
            }
            v = csub(v, cmul(a.phase[i], G0(sqrt(r2), a.k, a.ki)));
        }
        out[e] = v;
    }
}

__global__ void far_place_kernel(const double2* ftab, double2* X, int nf0, int nf1, int nf2, int L0, int L1, int L2,
                                 double scale) {
    const long long total = (long long)L0 * L1 * L2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int i0 = (int)(e % L0), i1 = (int)((e / L0) % L1), i2 = (int)(e / ((long long)L0 * L1));
        const int nf[3] = {nf0, nf1, nf2}, L[3] = {L0, L1, L2}, ii[3] = {i0, i1, i2};
        int t[3];
        bool used = true;
        for (int d = 0; d < 3; ++d) {
            int dl;
            if (ii[d] <= nf[d] - 1) dl = ii[d];
            else if (ii[d] >= L[d] - (nf[d] - 1)) dl = ii[d] - L[d];
            else { used = false; dl = 0; }
            t[d] = dl + nf[d] - 1;
        }
        double2 v = make_double2(0.0, 0.0);
        if (used) {
            const long long w0 = 2 * nf0 - 1, w1 = 2 * nf1 - 1;
            v = ftab[(t[2] * w1 + t[1]) * w0 + t[0]];
            v.x *= scale;
            v.y *= scale;
        }
        X[e] = v;
    }
}

int nextpow2(int v) {
    int p = 16;
    while (p < v) p *= 2;
    return p;
}

}  // namespace

int pim_fft_len(int n) { return nextpow2(2 * n - 1); }

pim_status build_near_spectrum(pim_plan P, cudaStream_t s) {
    FftGeom& g = P->ng;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = P->n[d];
        g.L[d] = nextpow2(2 * P->n[d] - 1);
    }
    const long long tot = (long long)g.L[0] * g.L[1] * g.L[2];
    double2* X = nullptr;
    int* dimg = nullptr;
    double2* dph = nullptr;
    pim_status st;
    if ((st = pim_alloc(P, (void**)&X, tot * sizeof(double2))) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&dimg, sizeof(int) * 3 * P->nimg)) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&dph, sizeof(double2) * P->nimg)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(dimg, P->img, sizeof(int) * 3 * P->nimg, cudaMemcpyHostToDevice, s));
    PIM_CK(cudaMemcpyAsync(dph, P->phase, sizeof(double2) * P->nimg, cudaMemcpyHostToDevice, s));
    NearArgs a{};
    for (int d = 0; d < 3; ++d) { a.n[d] = g.n[d]; a.L[d] = g.L[d]; a.h[d] = P->h[d]; }
    a.k = P->k;
    a.ki = P->ki;
    a.nimg = P->nimg;
    a.img = dimg;
    a.phase = dph;
    near_table_kernel<<<1024, 256, 0, s>>>(a, X);
    PIM_CK(cudaGetLastError());
    if ((st = fft3_forward_full<double>(P, g, X, nullptr, s)) != PIM_OK) return st;
    const double scale = 1.0 / (double)tot;
    const size_t esz = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
    // K(delta) is even along a non-periodic axis (no images there) and along
    // a periodic axis without phase shift (images i and -i weigh the same),
    // and so is its spectrum: keep frequencies 0..L/2 of those axes
    g.fold = 0;
    for (int d = 0; d < 3; ++d) {
        const bool even = !((P->pmask >> d) & 1u) || (P->k0[d] == 0.0 && P->k0i[d] == 0.0);
        if (even) g.fold |= 1 << d;
        g.S[d] = even ? g.L[d] / 2 + 1 : g.L[d];
    }
    const long long stot = (long long)g.S[0] * g.S[1] * g.S[2];
    if ((st = pim_alloc(P, &P->spec, stot * esz)) != PIM_OK) return st;
    if (P->prec == PIM_FP64)
        fold_convert_kernel<double><<<1024, 256, 0, s>>>(X, (double2*)P->spec, g.L[0], g.L[1], g.S[0], g.S[1], g.S[2],
                                                         scale);
    else
        fold_convert_kernel<float><<<1024, 256, 0, s>>>(X, (float2*)P->spec, g.L[0], g.L[1], g.S[0], g.S[1], g.S[2],
                                                        scale);
    PIM_CK(cudaGetLastError());
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, X, tot * sizeof(double2));
    pim_free(P, dimg, sizeof(int) * 3 * P->nimg);
    pim_free(P, dph, sizeof(double2) * P->nimg);
    return PIM_OK;
}

// The anomaly check with complex k or phase shift: a Floquet mode whose
// k_z^2 (k_rho^2) vanishes, or a vanishing denominator of Eq. pgf_3's z-image
// factor, in complex arithmetic.
static bool wood_anomaly_c(pim_plan P, const double* Lc, const double* k0r, const double* k0i) {
    using C = std::complex<double>;
    const C k(P->k, P->ki), kk = k * k;
    const C k0[3] = {C(k0r[0], k0i[0]), C(k0r[1], k0i[1]), C(k0r[2], k0i[2])};
    double scale = std::norm(k);
    for (int d = 0; d < P->npd && d < 2; ++d) scale = fmax(scale, pow(2.0 * PI / Lc[d], 2));
    const int M = (int)ceil((std::abs(k) + std::abs(k0[0])) * Lc[0] / (2.0 * PI)) + 2;
    if (P->npd == 1) {
        for (int m = -M; m <= M; ++m) {
            const C kx = k0[0] + 2.0 * PI * m / Lc[0];
            if (std::abs(kk - kx * kx) <= 1e-8 * scale) return true;
        }
        return false;
    }
    const int N = (int)ceil((std::abs(k) + std::abs(k0[1])) * Lc[1] / (2.0 * PI)) + 2;
    for (int m = -M; m <= M; ++m)
        for (int n = -N; n <= N; ++n) {
            const C kx = k0[0] + 2.0 * PI * m / Lc[0], ky = k0[1] + 2.0 * PI * n / Lc[1];
            const C r = kk - kx * kx - ky * ky;
            if (std::abs(r) <= 1e-8 * scale) return true;
            if (P->npd == 3) {
                C kz = std::sqrt(r);
                if (kz.imag() > 0.0) kz = -kz;
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const C e = std::exp(C(0.0, -1.0) * (kz + (double)sgn * k0[2]) * Lc[2]);
                    if (std::abs(1.0 - e) < 1e-9) return true;
                }
            }
        }
    return false;
}

// Rayleigh-Wood anomaly check (Sec. 2 after Eq. pgf): a Floquet mode with
// k_z = 0 (2D, 3D) or k_rho = 0 (1D), or a vanishing denominator of the
// z-image factor of Eq. pgf_3.
static bool wood_anomaly(pim_plan P, const double* Lc, const double* k0c) {
    if (P->npsp) return false;
    const double k = P->k;
    double scale = k * k;
    for (int d = 0; d < P->npd && d < 2; ++d) scale = fmax(scale, pow(2.0 * PI / Lc[d], 2));
    const int M = (int)ceil((k + fabs(k0c[0])) * Lc[0] / (2.0 * PI)) + 2;
    if (P->npd == 1) {
        for (int m = -M; m <= M; ++m) {
            const double kx = k0c[0] + 2.0 * PI * m / Lc[0];
            if (fabs(k * k - kx * kx) <= 1e-8 * scale) return true;
        }
        return false;
    }
    const int N = (int)ceil((k + fabs(k0c[1])) * Lc[1] / (2.0 * PI)) + 2;
    for (int m = -M; m <= M; ++m)
        for (int n = -N; n <= N; ++n) {
            const double kx = k0c[0] + 2.0 * PI * m / Lc[0], ky = k0c[1] + 2.0 * PI * n / Lc[1];
            const double r = k * k - kx * kx - ky * ky;
            if (fabs(r) <= 1e-8 * scale) return true;
            if (P->npd == 3 && r > 0) {
                const double kz = sqrt(r);
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const double ph = (kz + sgn * k0c[2]) * Lc[2] / (2.0 * PI);
                    if (fabs(ph - round(ph)) < 1e-9) return true;
                }
            }
        }
    if (P->npd == 3 && k == 0.0) {
        // static with phase: the (0,0) mode's z factor needs kz0 L != 2 pi q
        // unless the transverse wavenumber is nonzero (kz = -j|kt| then).
        const double ph = k0c[2] * Lc[2] / (2.0 * PI);
        const double tx = k0c[0] * Lc[0] / (2.0 * PI), ty = k0c[1] * Lc[1] / (2.0 * PI);
        if (fabs(tx - round(tx)) < 1e-12 && fabs(ty - round(ty)) < 1e-12 && fabs(ph - round(ph)) < 1e-12) return true;
    }
    return false;
}

pim_status build_far_table(pim_plan P, cudaStream_t s) {
    if (!P->has_far) return PIM_OK;
    FarArgs a{};
    int pc = 0;
    for (int d = 0; d < 3; ++d)
        if (P->pmask & (1u << d)) a.perm[pc++] = d;
    for (int d = 0; d < 3; ++d)
        if (!(P->pmask & (1u << d))) a.perm[pc++] = d;
    for (int d = 0; d < 3; ++d) {
        a.nf[d] = P->nf[d];
        a.df[d] = P->df[d];
        a.Lc[d] = P->D[a.perm[d]];
        a.k0c[d] = P->k0[a.perm[d]];
        a.k0ci[d] = P->k0i[a.perm[d]];
        a.D[d] = P->D[d];
    }
    a.npd = P->npd;
    a.k = P->k;
    a.ki = P->ki;
    a.cplx = (P->ki != 0.0 || a.k0ci[0] != 0.0 || a.k0ci[1] != 0.0 || a.k0ci[2] != 0.0) ? 1 : 0;
    a.npsp = P->npsp ? 1 : 0;
    auto anomaly = [&](const double* Lc, const double* kr, const double* ki) {
        return a.cplx ? wood_anomaly_c(P, Lc, kr, ki) : wood_anomaly(P, Lc, kr);
    };
    if (anomaly(a.Lc, a.k0c, a.k0ci)) {
        pim_set_error("Rayleigh-Wood anomaly: a Floquet mode has k_z (or k_rho) = 0 for these k, k0, L");
        return PIM_ERR_ANOMALY;
    }
    // 3D lattice: the axes that may serve as the series' z axis (z itself
    // always can, having passed the check above)
    a.zaxes = 1 << 2;
    if (P->npd == 3)
        for (int c = 0; c < 2; ++c) {
            const int c1 = c == 0 ? 1 : 0, c2 = 2;
            const double Lr[3] = {a.Lc[c1], a.Lc[c2], a.Lc[c]};
            const double kr[3] = {a.k0c[c1], a.k0c[c2], a.k0c[c]};
            const double kim[3] = {a.k0ci[c1], a.k0ci[c2], a.k0ci[c]};
            if (!anomaly(Lr, kr, kim)) a.zaxes |= 1 << c;
        }
    pim_status st;
    int* dimg = nullptr;
    double2* dph = nullptr;
    if ((st = pim_alloc(P, (void**)&dimg, sizeof(int) * 3 * P->nimg)) != PIM_OK) return st;
    if ((st = pim_alloc(P, (void**)&dph, sizeof(double2) * P->nimg)) != PIM_OK) return st;
    PIM_CK(cudaMemcpyAsync(dimg, P->img, sizeof(int) * 3 * P->nimg, cudaMemcpyHostToDevice, s));
    PIM_CK(cudaMemcpyAsync(dph, P->phase, sizeof(double2) * P->nimg, cudaMemcpyHostToDevice, s));
    a.nimg = P->nimg;
    a.img = dimg;
    a.phase = dph;
    a.bad = P->dstatus;  // zero at plan creation
    const int ntab = (2 * P->nf[0] - 1) * (2 * P->nf[1] - 1) * (2 * P->nf[2] - 1);
    if ((st = pim_alloc(P, (void**)&P->ftab, sizeof(double2) * ntab)) != PIM_OK) return st;
    far_table_kernel<<<ntab, FAR_NT, 0, s>>>(a, P->ftab);
    PIM_CK(cudaGetLastError());
    if (a.cplx && P->npd == 1) {
        int bad = 0;
        PIM_CK(cudaMemcpyAsync(&bad, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
        PIM_CK(cudaStreamSynchronize(s));
        PIM_CK(cudaMemsetAsync(P->dstatus, 0, sizeof(int), s));
        if (bad) {
            pim_set_error("1D series with complex k or k0: a Hankel-function argument of modulus between 6 and "
                          "20 lies within 0.17 rad of the real axis (a weakly lossy propagating mode); not supported");
            return PIM_ERR_UNSUPPORTED;
        }
    }
    // far spectrum for the grid sum of Eq. 8 by zero-padded FFT
    FftGeom& g = P->fg;
    for (int d = 0; d < 3; ++d) {
        g.n[d] = P->nf[d];
        g.L[d] = nextpow2(2 * P->nf[d] - 1);
    }
    const long long tot = (long long)g.L[0] * g.L[1] * g.L[2];
    if ((st = pim_alloc(P, (void**)&P->fspec, tot * sizeof(double2))) != PIM_OK) return st;
    far_place_kernel<<<256, 256, 0, s>>>(P->ftab, P->fspec, g.n[0], g.n[1], g.n[2], g.L[0], g.L[1], g.L[2],
                                         1.0 / (double)tot);
    PIM_CK(cudaGetLastError());
    if ((st = fft3_forward_full<double>(P, g, P->fspec, nullptr, s)) != PIM_OK) return st;
    PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, dimg, sizeof(int) * 3 * P->nimg);
    pim_free(P, dph, sizeof(double2) * P->nimg);
    return PIM_OK;
}
