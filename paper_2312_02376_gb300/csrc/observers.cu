// Observer points apart from the sources (the paper's accuracy test, Sec.
// 4.1: potentials evaluated at points that carry no source).  The plan holds
// the N sources and the M observers as one point set, sources first; an
// observer is a point of zero strength.  The rows of that operator at the
// observers, applied to [q; 0], are the potentials at the observers (Eq. 1
// with r_m an observer), and its source rows of the adjoint, applied to
// [0; v], are the adjoint of that map.  In the neutral static case the
// regularisation of Eq. neutral removes the mean over the sources only, and
// the adjoint projects its result on the sources' neutral subspace.
#include "pim_internal.cuh"

namespace {

bool dev_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// bytes of one value of the plan's data type (real for the static case
// without phase, complex otherwise)
size_t value_bytes(pim_plan P) {
    const size_t r = P->prec == PIM_FP64 ? sizeof(double) : sizeof(float);
    return P->real_data ? r : 2 * r;
}

constexpr int MEAN_NT = 256;

// One CTA per right-hand side r: the FP64 mean of x[0..N)[r] into mean[2r],
// mean[2r+1]; with check, the neutrality test of Eq. neutral
// (|sum x| <= tol sum |x|, else PIM_DEV_NOT_NEUTRAL in *status).
template <typename T, bool REAL>
__global__ void __launch_bounds__(MEAN_NT) src_mean_kernel(const T* x, long long N, int nrhs, double tol, int check,
                                                           double* mean, int* status) {
    __shared__ double sh[3][MEAN_NT];
    const int r = blockIdx.x;
    double a = 0.0, b = 0.0, c = 0.0;
    for (long long i = threadIdx.x; i < N; i += MEAN_NT) {
        const long long e = i * nrhs + r;
        const double re = REAL ? (double)x[e] : (double)x[2 * e], im = REAL ? 0.0 : (double)x[2 * e + 1];
        a += re;
        b += im;
        c += sqrt(re * re + im * im);
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    sh[2][threadIdx.x] = c;
    __syncthreads();
    for (int s = MEAN_NT / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            for (int k = 0; k < 3; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mean[2 * r] = N > 0 ? sh[0][0] / (double)N : 0.0;
        mean[2 * r + 1] = N > 0 ? sh[1][0] / (double)N : 0.0;
        if (check && sqrt(sh[0][0] * sh[0][0] + sh[1][0] * sh[1][0]) > tol * sh[2][0]) atomicOr(status, PIM_DEV_NOT_NEUTRAL);
    }
}

// x[0..N)[r] -= mean[r], formed in FP64
template <typename T, bool REAL>
__global__ void sub_mean_kernel(T* x, long long N, int nrhs, const double* mean) {
    const long long tot = N * nrhs;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % nrhs);
        if (REAL) {
            x[e] = (T)((double)x[e] - mean[2 * r]);
        } else {
            x[2 * e] = (T)((double)x[2 * e] - mean[2 * r]);
            x[2 * e + 1] = (T)((double)x[2 * e + 1] - mean[2 * r + 1]);
        }
    }
}

template <typename T>
void launch_mean(pim_plan P, const void* x, long long N, int nrhs, bool check, cudaStream_t s) {
    if (P->real_data)
        src_mean_kernel<T, true><<<nrhs, MEAN_NT, 0, s>>>((const T*)x, N, nrhs, P->neutral_tol, check ? 1 : 0,
                                                          P->obs_means, P->dstatus);
    else
        src_mean_kernel<T, false><<<nrhs, MEAN_NT, 0, s>>>((const T*)x, N, nrhs, P->neutral_tol, check ? 1 : 0,
                                                           P->obs_means, P->dstatus);
}

template <typename T>
void launch_sub(pim_plan P, void* x, long long N, int nrhs, cudaStream_t s) {
    const unsigned nb = (unsigned)std::min<long long>((N * nrhs + 255) / 256, 152 * 8);
    if (nb == 0) return;
    if (P->real_data) sub_mean_kernel<T, true><<<nb, 256, 0, s>>>((T*)x, N, nrhs, P->obs_means);
    else sub_mean_kernel<T, false><<<nb, 256, 0, s>>>((T*)x, N, nrhs, P->obs_means);
}

pim_status ensure_buffers(pim_plan P, size_t bytes, int nrhs) {
    pim_status st;
    if (P->obs_bytes < bytes) {
        pim_free(P, P->obs_q, P->obs_bytes);
        pim_free(P, P->obs_u, P->obs_bytes);
        P->obs_q = P->obs_u = nullptr;
        P->obs_bytes = 0;
        if ((st = pim_alloc(P, &P->obs_q, bytes)) != PIM_OK) return st;
        if ((st = pim_alloc(P, &P->obs_u, bytes)) != PIM_OK) return st;
        P->obs_bytes = bytes;
    }
    if (P->obs_nmeans < nrhs) {
        pim_free(P, P->obs_means, 2 * sizeof(double) * P->obs_nmeans);
        P->obs_means = nullptr;
        P->obs_nmeans = 0;
        if ((st = pim_alloc(P, (void**)&P->obs_means, 2 * sizeof(double) * nrhs)) != PIM_OK) return st;
        P->obs_nmeans = nrhs;
    }
    return PIM_OK;
}

pim_status observers_apply(pim_plan P, const void* in, void* out, int nrhs, void* stream, bool adj) {
    if (!P || !in || !out || nrhs < 1) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (P->nobs <= 0 || !P->pts.box_ptr) {
        pim_set_error("no observer points: call pim_set_points_observers first");
        return PIM_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const long long N = P->nsrc, M = P->nobs;
    const size_t vb = value_bytes(P), src_bytes = (size_t)N * nrhs * vb, obs_bytes = (size_t)M * nrhs * vb;
    pim_status st;
    if ((st = ensure_buffers(P, src_bytes + obs_bytes, nrhs)) != PIM_OK) return st;
    char* pq = (char*)P->obs_q;
    char* pu = (char*)P->obs_u;
    const bool fp64 = P->prec == PIM_FP64;
    if (!adj) {
        // [q; 0], the sources' mean removed in the neutral static case
        if (src_bytes) PIM_CK(cudaMemcpyAsync(pq, in, src_bytes, cudaMemcpyDefault, s));
        PIM_CK(cudaMemsetAsync(pq + src_bytes, 0, obs_bytes, s));
        if (P->npsp && N > 0) {
            if (fp64) {
                launch_mean<double>(P, pq, N, nrhs, true, s);
                launch_sub<double>(P, pq, N, nrhs, s);
            } else {
                launch_mean<float>(P, pq, N, nrhs, true, s);
                launch_sub<float>(P, pq, N, nrhs, s);
            }
            PIM_CK(cudaGetLastError());
        }
        if ((st = apply_run(P, pq, pu, nrhs, false, s)) != PIM_OK) return st;
        PIM_CK(cudaMemcpyAsync(out, pu + src_bytes, obs_bytes, cudaMemcpyDefault, s));
    } else {
        // [0; v]; the source rows of the result, projected on the sources'
        // neutral subspace in the neutral static case
        if (src_bytes) PIM_CK(cudaMemsetAsync(pq, 0, src_bytes, s));
        PIM_CK(cudaMemcpyAsync(pq + src_bytes, in, obs_bytes, cudaMemcpyDefault, s));
        if ((st = apply_run(P, pq, pu, nrhs, true, s)) != PIM_OK) return st;
        if (P->npsp && N > 0) {
            if (fp64) {
                launch_mean<double>(P, pu, N, nrhs, false, s);
                launch_sub<double>(P, pu, N, nrhs, s);
            } else {
                launch_mean<float>(P, pu, N, nrhs, false, s);
                launch_sub<float>(P, pu, N, nrhs, s);
            }
            PIM_CK(cudaGetLastError());
        }
        if (src_bytes) PIM_CK(cudaMemcpyAsync(out, pu, src_bytes, cudaMemcpyDefault, s));
    }
    if (!dev_ptr(in) || !dev_ptr(out)) PIM_CK(cudaStreamSynchronize(s));
    return PIM_OK;
}

}  // namespace

pim_status pim_set_points_observers(pim_plan P, int64_t N, const double* xyz, int64_t M, const double* obs) {
    if (!P || N < 0 || M < 1 || (N > 0 && !xyz) || !obs) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    double* all = nullptr;
    pim_status st;
    if ((st = pim_alloc(P, (void**)&all, 3 * (size_t)(N + M) * sizeof(double))) != PIM_OK) return st;
    if ((N > 0 && cudaMemcpy(all, xyz, 3 * (size_t)N * sizeof(double), cudaMemcpyDefault) != cudaSuccess) ||
        cudaMemcpy(all + 3 * N, obs, 3 * (size_t)M * sizeof(double), cudaMemcpyDefault) != cudaSuccess) {
        cudaGetLastError();
        pim_free(P, all, 3 * (size_t)(N + M) * sizeof(double));
        pim_set_error("copy of the point positions failed");
        return PIM_ERR_CUDA;
    }
    st = pim_set_points(P, N + M, all);
    pim_free(P, all, 3 * (size_t)(N + M) * sizeof(double));
    if (st != PIM_OK) return st;
    P->nsrc = N;
    P->nobs = M;
    return PIM_OK;
}

pim_status pim_apply_observers(pim_plan P, const void* q, void* u, int nrhs, void* stream) {
    return observers_apply(P, q, u, nrhs, stream, false);
}

pim_status pim_apply_observers_adjoint(pim_plan P, const void* v, void* w, int nrhs, void* stream) {
    return observers_apply(P, v, w, nrhs, stream, true);
}

void observers_free(pim_plan P) {
    pim_free(P, P->obs_q, P->obs_bytes);
    pim_free(P, P->obs_u, P->obs_bytes);
    pim_free(P, P->obs_means, 2 * sizeof(double) * P->obs_nmeans);
    P->obs_q = P->obs_u = nullptr;
    P->obs_means = nullptr;
    P->obs_bytes = 0;
    P->obs_nmeans = 0;
}
