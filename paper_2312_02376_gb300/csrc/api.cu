// C ABI of libpim (include/pim.h): plan life cycle, argument checks,
// memory accounting and host-pointer staging.
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "pim_internal.cuh"

namespace {
thread_local std::string g_last_error;

double now_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

size_t grid_elem(pim_plan P) { return P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2); }
size_t data_elem(pim_plan P) {
    const size_t r = P->prec == PIM_FP64 ? sizeof(double) : sizeof(float);
    return P->real_data ? r : 2 * r;
}
}  // namespace

void pim_set_error(const std::string& msg) { g_last_error = msg; }

int far_stream_priority() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return greatest;
}

int lf_stream_priority() {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return least;
}

pim_status pim_alloc(pim_plan P, void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (bytes == 0) return PIM_OK;
    if (P->mem_cap && P->bytes + bytes > P->mem_cap) {
        pim_set_error("plan memory cap exceeded");
        return PIM_ERR_OOM;
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        pim_set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e));
        return PIM_ERR_OOM;
    }
    P->bytes += bytes;
    return PIM_OK;
}

void prof_mark(pim_plan P, int stage, int which, cudaStream_t s) {
    if (!P->prof_on || P->prof_next >= pim_plan_s::PROF_RING) return;
    const int slot = P->prof_next;
    cudaEventRecord(P->prof_ev[(slot * PIM_NUM_STAGES + stage) * 2 + which], s);
    if (which == 1) P->prof_mask[slot] |= (unsigned short)(1u << stage);
}

void pim_free(pim_plan P, void* ptr, size_t bytes) {
    if (!ptr) return;
    cudaFree(ptr);
    P->bytes -= bytes;
}

static void free_grad_buffers(pim_plan P) {
    const size_t ge = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t G = (size_t)P->n[0] * P->n[1] * P->n[2];
    const size_t Gf = P->has_far ? (size_t)P->nf[0] * P->nf[1] * P->nf[2] : 0;
    pim_free(P, P->gD, G * ge);
    pim_free(P, P->gsrt, (size_t)std::max<int64_t>(1, P->pts.N) * ge);
    pim_free(P, P->fD, Gf * sizeof(double2));
    pim_free(P, P->fU, Gf * ge);
    pim_free(P, P->fV, Gf * ge);
    P->gD = P->gsrt = P->fU = P->fV = nullptr;
    P->fD = nullptr;
}

static pim_status position_grad(pim_plan P, const void* q, const void* g, double* grad, int nrhs, void* stream,
                                bool reuse);

// Buffers of the position gradient: V, the sorted g, the far charges and
// both far potentials (kept between applies for pim_position_grad_reuse).
pim_status alloc_grad_buffers(pim_plan P) {
    if (P->gsrt) return PIM_OK;
    const size_t ge = grid_elem(P);
    const size_t G = (size_t)P->n[0] * P->n[1] * P->n[2];
    const size_t Gf = P->has_far ? (size_t)P->nf[0] * P->nf[1] * P->nf[2] : 0;
    pim_status st;
    if ((st = pim_alloc(P, &P->gD, G * ge)) != PIM_OK) return st;
    if ((st = pim_alloc(P, &P->gsrt, (size_t)std::max<int64_t>(1, P->pts.N) * ge)) != PIM_OK) return st;
    if (Gf) {
        if ((st = pim_alloc(P, (void**)&P->fD, Gf * sizeof(double2))) != PIM_OK) return st;
        if ((st = pim_alloc(P, &P->fU, Gf * ge)) != PIM_OK) return st;
        if ((st = pim_alloc(P, &P->fV, Gf * ge)) != PIM_OK) return st;
    }
    return PIM_OK;
}

extern "C" {

const char* pim_last_error(void) { return g_last_error.c_str(); }

void pim_options_default(pim_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->far_p = -1;
    o->corr_radius = -1;
    o->corr_cube = 0;
    o->corr_mode = PIM_CORR_COMPACT;
    o->neutral_tol = 1e-6;
    o->series_tol = 1e-16;
    o->mem_cap = 0;
    o->autotune = 1;
    o->with_gradient = 0;
    o->corr_split = 10;
    o->gather_variant = -1;
    o->corr_listfree = -1;
    o->lf_tensor_cores = 1;
    o->k_imag = 0.0;
    for (int d = 0; d < 3; ++d) o->k0_imag[d] = 0.0;
}

const char* pim_status_string(pim_status s) {
    switch (s) {
        case PIM_OK: return "PIM_OK";
        case PIM_ERR_ARG: return "PIM_ERR_ARG";
        case PIM_ERR_UNSUPPORTED: return "PIM_ERR_UNSUPPORTED";
        case PIM_ERR_ANOMALY: return "PIM_ERR_ANOMALY";
        case PIM_ERR_NOT_NEUTRAL: return "PIM_ERR_NOT_NEUTRAL";
        case PIM_ERR_OUT_OF_CELL: return "PIM_ERR_OUT_OF_CELL";
        case PIM_ERR_STATE: return "PIM_ERR_STATE";
        case PIM_ERR_OOM: return "PIM_ERR_OOM";
        case PIM_ERR_CUDA: return "PIM_ERR_CUDA";
        case PIM_ERR_TIMEOUT: return "PIM_ERR_TIMEOUT";
        case PIM_ERR_DEVICE: return "PIM_ERR_DEVICE";
    }
    return "unknown";
}

void pim_destroy(pim_plan P) {
    if (!P) return;
    cudaDeviceSynchronize();
    batch_forget(P);
    lanes_free(P);
    observers_free(P);
    if (P->lane_fork) cudaEventDestroy(P->lane_fork);
    {
        const size_t gq = grid_elem(P) * (size_t)P->pts.N;
        pim_free(P, P->qs, gq);
        pim_free(P, P->us, gq);
        pim_free(P, P->ufp, gq);
        pim_free(P, P->ulf, P->ulf ? gq : 0);
        pim_free(P, P->hq, P->stage_bytes);
        pim_free(P, P->hu, P->stage_bytes);
    }
    points_free(P);
    const size_t ge = grid_elem(P);
    const long long G = (long long)P->n[0] * P->n[1] * P->n[2];
    const long long Gs = (long long)P->ng.S[0] * P->ng.S[1] * P->ng.S[2];
    pim_free(P, P->spec, Gs * ge);
    pim_free(P, P->gA, G * ge);
    pim_free(P, P->gB, (long long)P->n[2] * P->n[1] * P->ng.L[0] * ge);
    pim_free(P, P->gC, (long long)P->n[2] * P->ng.L[1] * P->ng.L[0] * ge);
    if (P->has_far) {
        const long long Gf = (long long)P->nf[0] * P->nf[1] * P->nf[2];
        const long long Wf = (long long)(2 * P->nf[0] - 1) * (2 * P->nf[1] - 1) * (2 * P->nf[2] - 1);
        pim_free(P, P->ftab, Wf * sizeof(double2));
        pim_free(P, P->fspec, (long long)P->fg.L[0] * P->fg.L[1] * P->fg.L[2] * sizeof(double2));
        pim_free(P, P->fA, Gf * sizeof(double2));
        pim_free(P, P->fB, (long long)P->nf[2] * P->nf[1] * P->fg.L[0] * sizeof(double2));
        pim_free(P, P->fC, (long long)P->nf[2] * P->fg.L[1] * P->fg.L[0] * sizeof(double2));
        pim_free(P, P->fpart, (size_t)P->far_chunks * Gf * ge);
    }
    free_grad_buffers(P);
    pim_free(P, P->qsall, P->qsall_bytes);
    pim_free(P, P->dmeans, 2 * 128 * sizeof(double));
    pim_free(P, P->tw32, 2048 * sizeof(float2));
    pim_free(P, P->tw64, 2048 * sizeof(double2));
    pim_free(P, P->dsum, sizeof(double) * (4 + 3 * PIM_RED_BLOCKS));
    pim_free(P, P->dphase, 2 * (sizeof(double2) + sizeof(float4)) * PIM_MAX_IMAGES);
    pim_free(P, P->dstatus, sizeof(int));
    pim_free(P, P->lfnext, sizeof(unsigned long long) * (pim_plan_s::RHS_LANES + 1));
    if (P->prof_ev) {
        for (int i = 0; i < pim_plan_s::PROF_RING * PIM_NUM_STAGES * 2; ++i) cudaEventDestroy(P->prof_ev[i]);
        delete[] P->prof_ev;
    }
    if (P->s_far) cudaStreamDestroy(P->s_far);
    if (P->s_main) cudaStreamDestroy(P->s_main);
    if (P->s_lf) cudaStreamDestroy(P->s_lf);
    if (P->ev_fork) cudaEventDestroy(P->ev_fork);
    if (P->ev_join) cudaEventDestroy(P->ev_join);
    if (P->ev_lf_fork) cudaEventDestroy(P->ev_lf_fork);
    if (P->ev_lf_mom) cudaEventDestroy(P->ev_lf_mom);
    if (P->ev_lf_join) cudaEventDestroy(P->ev_lf_join);
    delete P;
}

pim_status pim_plan_create(pim_plan* out, const double lattice[9], unsigned pmask, double k, const double k0[3],
                           const double h[3], int p, int near_layers, pim_precision prec, const pim_options* opt,
                           void* stream) {
    const double t0 = now_ms();
    if (!out || !lattice || !k0 || !h) {
        pim_set_error("null argument");
        return PIM_ERR_ARG;
    }
    *out = nullptr;
    pim_options o;
    if (opt) o = *opt;
    else pim_options_default(&o);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i != j && lattice[3 * i + j] != 0.0) {
                pim_set_error("only rectangular (diagonal) lattices are supported");
                return PIM_ERR_UNSUPPORTED;
            }
    if (pmask > 7u || !(k >= 0.0) || !std::isfinite(k) || near_layers < 0 || (prec != PIM_FP64 && prec != PIM_FP32_MIXED)) {
        pim_set_error("invalid periodic mask, wavenumber, layer count or precision");
        return PIM_ERR_ARG;
    }
    if (p < 2 || p > 4) {
        pim_set_error("interpolation degree p must be 2, 3 or 4 on the GPU path");
        return PIM_ERR_UNSUPPORTED;
    }
    const bool cplx = o.k_imag != 0.0 || o.k0_imag[0] != 0.0 || o.k0_imag[1] != 0.0 || o.k0_imag[2] != 0.0;
    if (!(o.k_imag <= 0.0) || !std::isfinite(o.k0_imag[0]) || !std::isfinite(o.k0_imag[1]) ||
        !std::isfinite(o.k0_imag[2])) {
        pim_set_error("Im k must be <= 0 (a lossy medium) and the phase shift finite");
        return PIM_ERR_ARG;
    }
    if (cplx && o.with_gradient) {
        pim_set_error("the position gradient needs a real k and k0");
        return PIM_ERR_UNSUPPORTED;
    }
    pim_plan P = new pim_plan_s();
    auto fail = [&](pim_status st) {
        pim_destroy(P);
        return st;
    };
    P->pmask = pmask;
    P->k = k;
    P->ki = o.k_imag;
    P->p = p;
    P->layers = near_layers;
    P->prec = prec;
    P->mem_cap = o.mem_cap;
    P->autotune = o.autotune ? 1 : 0;
    P->with_gradient = o.with_gradient ? 1 : 0;
    P->lf_tc = o.lf_tensor_cores ? 1 : 0;
    P->force_variant = o.gather_variant;
    // the list-free kernels' polynomials in r^2 assume a real k
    P->lf_min_work = P->with_gradient || o.k_imag != 0.0 ? 0 : (o.corr_listfree < 0 ? 131072 : o.corr_listfree);
    P->neutral_tol = o.neutral_tol > 0 ? o.neutral_tol : 1e-6;
    P->series_tol = o.series_tol > 0 ? o.series_tol : 1e-16;
    P->npd = 0;
    for (int d = 0; d < 3; ++d) {
        P->D[d] = lattice[4 * d];
        P->k0[d] = k0[d];
        P->k0i[d] = o.k0_imag[d];
        if (!(P->D[d] > 0.0) || !std::isfinite(P->D[d]) || !(h[d] > 0.0) || !std::isfinite(k0[d])) {
            pim_set_error("cell extents and grid spacings must be positive and finite");
            return fail(PIM_ERR_ARG);
        }
        const bool per = (pmask >> d) & 1u;
        if (per) P->npd++;
        if (!per && (k0[d] != 0.0 || o.k0_imag[d] != 0.0)) {
            pim_set_error("phase shift on a non-periodic axis");
            return fail(PIM_ERR_ARG);
        }
        const double steps = P->D[d] / h[d];
        const double rs = std::round(steps);
        if (std::fabs(steps - rs) > 1e-9 * std::max(1.0, steps) || rs < 1) {
            pim_set_error("D/h must be an integer on every axis");
            return fail(PIM_ERR_ARG);
        }
        P->n[d] = (int)rs + 1;
        P->nb[d] = (p & 1) ? P->n[d] - 1 : P->n[d];
        P->h[d] = P->D[d] / rs;
        if (P->n[d] < p + 1 || P->n[d] > 1024) {
            pim_set_error("near grid must have p+1 .. 1024 nodes per axis");
            return fail(PIM_ERR_ARG);
        }
    }
    const bool k_zero = k == 0.0 && k0[0] == 0.0 && k0[1] == 0.0 && k0[2] == 0.0 && !cplx;
    P->npsp = P->npd > 0 && k_zero;
    P->real_data = k_zero;
    P->b = o.corr_radius >= 0 ? o.corr_radius : p + 1;
    P->cube = o.corr_cube ? 1 : 0;
    P->corr_mode = prec == PIM_FP64 ? PIM_CORR_FP64 : o.corr_mode;
    if (P->corr_mode < 0 || P->corr_mode > 3) {
        pim_set_error("invalid correction mode");
        return fail(PIM_ERR_ARG);
    }
    if (o.corr_split < 0 || o.corr_split > 30) {
        pim_set_error("corr_split outside [0, 30]");
        return fail(PIM_ERR_ARG);
    }
    P->corr_split = o.corr_split;
    // near images (Eq. 4)
    P->nimg = 0;
    const int Lr = near_layers;
    const int lx = (pmask & 1) ? Lr : 0, ly = (pmask & 2) ? Lr : 0, lz = (pmask & 4) ? Lr : 0;
    if ((2 * lx + 1) * (2 * ly + 1) * (2 * lz + 1) > PIM_MAX_IMAGES) {
        pim_set_error("too many near images");
        return fail(PIM_ERR_UNSUPPORTED);
    }
    for (int iz = -lz; iz <= lz; ++iz)
        for (int iy = -ly; iy <= ly; ++iy)
            for (int ix = -lx; ix <= lx; ++ix) {
                int* v = P->img[P->nimg];
                v[0] = ix; v[1] = iy; v[2] = iz;
                // exp(-j k0.a), k0 = k0 + j k0i: modulus exp(k0i.a), angle -k0.a
                const double th = -(k0[0] * ix * P->D[0] + k0[1] * iy * P->D[1] + k0[2] * iz * P->D[2]);
                const double lm = o.k0_imag[0] * ix * P->D[0] + o.k0_imag[1] * iy * P->D[1] +
                                  o.k0_imag[2] * iz * P->D[2];
                const double mag = lm != 0.0 ? std::exp(lm) : 1.0;
                P->phase[P->nimg] = make_double2(mag * std::cos(th), mag * std::sin(th));
                // the adjoint's phase exp(-j conj(k0).a): modulus exp(-k0i.a)
                P->phase_adj[P->nimg] = make_double2(std::cos(th) / mag, std::sin(th) / mag);
                P->nimg++;
            }
    if (P->nimg > (1 << (32 - PIM_COL_BITS))) return fail(PIM_ERR_UNSUPPORTED);
    // far grids (Eq. grid)
    P->has_far = P->npd > 0;
    P->pf = o.far_p >= 0 ? o.far_p : p;
    for (int d = 0; d < 3; ++d) {
        P->nf[d] = o.far_n[d] > 0 ? o.far_n[d] : std::max(10, (int)std::ceil(4.0 * std::hypot(k, P->ki) * P->D[d]));
        P->df[d] = P->D[d] / P->nf[d];
        if (P->has_far && (P->nf[d] < P->pf + 1 || P->nf[d] > 512)) {
            pim_set_error("far grid must have p_f+1 .. 512 nodes per axis");
            return fail(PIM_ERR_ARG);
        }
    }
    if (P->has_far && (P->pf < 2 || P->pf > 6)) {
        pim_set_error("far degree must be 2..6");
        return fail(PIM_ERR_UNSUPPORTED);
    }
    cudaStream_t s = (cudaStream_t)stream;
    pim_status st;
    // the far zone's stream takes the highest priority: its short chain ends
    // with the far interpolation, which then runs ahead of the pending blocks
    // of the near gather instead of after them
    // the list-free exact kernel's stream the lowest: its compute-bound blocks
    // fill the SMs that the memory-bound near path leaves idle
    if (cudaStreamCreateWithPriority(&P->s_far, cudaStreamNonBlocking, far_stream_priority()) != cudaSuccess ||
        cudaStreamCreateWithPriority(&P->s_lf, cudaStreamNonBlocking, lf_stream_priority()) != cudaSuccess ||
        cudaStreamCreateWithFlags(&P->s_main, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_lf_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_lf_mom, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->ev_lf_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        pim_set_error("stream or event creation failed");
        return fail(PIM_ERR_CUDA);
    }
    if ((st = pim_alloc(P, (void**)&P->dstatus, sizeof(int))) != PIM_OK) return fail(st);
    if ((st = pim_alloc(P, (void**)&P->lfnext, sizeof(unsigned long long) * (pim_plan_s::RHS_LANES + 1))) != PIM_OK)
        return fail(st);
    if ((st = pim_alloc(P, (void**)&P->dsum, sizeof(double) * (4 + 3 * PIM_RED_BLOCKS))) != PIM_OK) return fail(st);
    if ((st = pim_alloc(P, (void**)&P->dphase, 2 * (sizeof(double2) + sizeof(float4)) * PIM_MAX_IMAGES)) != PIM_OK)
        return fail(st);
    P->dphasedf = reinterpret_cast<float4*>(P->dphase + PIM_MAX_IMAGES);
    P->dphase_adj = reinterpret_cast<double2*>(P->dphasedf + PIM_MAX_IMAGES);
    P->dphasedf_adj = reinterpret_cast<float4*>(P->dphase_adj + PIM_MAX_IMAGES);
    float4 phdf[PIM_MAX_IMAGES], phdfa[PIM_MAX_IMAGES];
    auto split = [](double2 v) {
        const float rh = (float)v.x, ih = (float)v.y;
        return make_float4(rh, (float)(v.x - (double)rh), ih, (float)(v.y - (double)ih));
    };
    for (int i = 0; i < P->nimg; ++i) {
        phdf[i] = split(P->phase[i]);
        phdfa[i] = split(P->phase_adj[i]);
    }
    if (cudaMemset(P->dstatus, 0, sizeof(int)) != cudaSuccess ||
        cudaMemcpy(P->dphase, P->phase, sizeof(double2) * P->nimg, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->dphasedf, phdf, sizeof(float4) * P->nimg, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->dphase_adj, P->phase_adj, sizeof(double2) * P->nimg, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(P->dphasedf_adj, phdfa, sizeof(float4) * P->nimg, cudaMemcpyHostToDevice) != cudaSuccess) {
        pim_set_error("initial copies failed");
        return fail(PIM_ERR_CUDA);
    }
    if ((st = fft_make_twiddles(P)) != PIM_OK) return fail(st);
    if ((st = build_near_spectrum(P, s)) != PIM_OK) return fail(st);
    const size_t ge = grid_elem(P);
    const long long G = (long long)P->n[0] * P->n[1] * P->n[2];
    if ((st = pim_alloc(P, &P->gA, G * ge)) != PIM_OK) return fail(st);
    if ((st = pim_alloc(P, &P->gB, (long long)P->n[2] * P->n[1] * P->ng.L[0] * ge)) != PIM_OK) return fail(st);
    if ((st = pim_alloc(P, &P->gC, (long long)P->n[2] * P->ng.L[1] * P->ng.L[0] * ge)) != PIM_OK) return fail(st);
    if (P->has_far) {
        if ((st = build_far_table(P, s)) != PIM_OK) return fail(st);
        const long long Gf = (long long)P->nf[0] * P->nf[1] * P->nf[2];
        // far grids that do not fit in shared memory once per CTA are spread
        // by z-windows (no per-CTA partial grids)
        P->far_window = Gf * 2 * (prec == PIM_FP64 ? 8 : 4) > 200 * 1024;
        P->far_chunks = P->far_window ? 0 : 304;
        if ((st = pim_alloc(P, (void**)&P->fA, Gf * sizeof(double2))) != PIM_OK) return fail(st);
        if ((st = pim_alloc(P, (void**)&P->fB, (long long)P->nf[2] * P->nf[1] * P->fg.L[0] * sizeof(double2))) != PIM_OK)
            return fail(st);
        if ((st = pim_alloc(P, (void**)&P->fC, (long long)P->nf[2] * P->fg.L[1] * P->fg.L[0] * sizeof(double2))) !=
            PIM_OK)
            return fail(st);
        if (!P->far_window && (st = pim_alloc(P, &P->fpart, (size_t)P->far_chunks * Gf * ge)) != PIM_OK)
            return fail(st);
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        pim_set_error(cudaGetErrorString(cudaGetLastError()));
        return fail(PIM_ERR_CUDA);
    }
    P->plan_ms = now_ms() - t0;
    *out = P;
    return PIM_OK;
}

pim_status pim_set_points(pim_plan P, int64_t N, const double* xyz) {
    if (!P || N < 0 || (N > 0 && !xyz)) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (N > (int64_t)PIM_COL_MASK) {
        pim_set_error("too many points");
        return PIM_ERR_UNSUPPORTED;
    }
    const double t0 = now_ms();
    cudaDeviceSynchronize();
    batch_forget(P);
    lanes_free(P);  // their sizes depend on the points
    observers_free(P);
    P->nsrc = N;    // pim_set_points_observers sets the split after this call
    P->nobs = 0;
    const size_t ge = grid_elem(P);
    if (P->pts.N > 0 || P->pts.box_ptr) {
        free_grad_buffers(P);
        pim_free(P, P->qsall, P->qsall_bytes);
        P->qsall = nullptr;
        P->qsall_bytes = 0;
        pim_free(P, P->qs, (size_t)P->pts.N * ge);
        pim_free(P, P->us, (size_t)P->pts.N * ge);
        pim_free(P, P->ufp, (size_t)P->pts.N * ge);
        pim_free(P, P->ulf, P->ulf ? (size_t)P->pts.N * ge : 0);
        P->qs = P->us = P->ufp = P->ulf = nullptr;
        points_free(P);
    }
    const double* dx = xyz;
    double* tmp = nullptr;
    pim_status st;
    if (N > 0 && !is_device_ptr(xyz)) {
        if ((st = pim_alloc(P, (void**)&tmp, 3 * N * sizeof(double))) != PIM_OK) return st;
        PIM_CK(cudaMemcpy(tmp, xyz, 3 * N * sizeof(double), cudaMemcpyHostToDevice));
        dx = tmp;
    }
    P->pot_valid = 0;
    st = points_build(P, N, dx, 0);
    if (tmp) pim_free(P, tmp, 3 * N * sizeof(double));
    if (st != PIM_OK) {
        points_free(P);
        return st;
    }
    if ((st = pim_alloc(P, &P->qs, (size_t)N * ge)) != PIM_OK) return st;
    if ((st = pim_alloc(P, &P->us, (size_t)N * ge)) != PIM_OK) return st;
    if (P->has_far && (st = pim_alloc(P, &P->ufp, (size_t)N * ge)) != PIM_OK) return st;
    if (P->pts.nlf > 0 && (st = pim_alloc(P, &P->ulf, (size_t)N * ge)) != PIM_OK) return st;
    if (P->with_gradient && (st = alloc_grad_buffers(P)) != PIM_OK) return st;
    P->gather_variant = 0;
    if (P->force_variant >= 0) {
        if (P->force_variant >= gather_variant_count(P)) return PIM_ERR_ARG;
        P->gather_variant = P->force_variant;
    } else if (P->autotune && N > 0 && (st = apply_autotune(P, 0)) != PIM_OK) {
        return st;
    }
    P->pot_valid = 0;  // the autotuner's applies are not the caller's
    PIM_CK(cudaDeviceSynchronize());
    P->points_ms = now_ms() - t0;
    return PIM_OK;
}

static pim_status apply_common(pim_plan P, const void* q, void* u, int nrhs, void* stream, bool adj) {
    if (!P || !q || !u || nrhs < 1) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (!P->pts.box_ptr) {
        pim_set_error("apply before pim_set_points");
        return PIM_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)P->pts.N * nrhs * data_elem(P);
    const bool hq = !is_device_ptr(q), hu = !is_device_ptr(u);
    if (!hq && !hu) return apply_run(P, q, u, nrhs, adj, s);
    pim_status st;
    if (P->stage_bytes < bytes) {
        pim_free(P, P->hq, P->stage_bytes);
        pim_free(P, P->hu, P->stage_bytes);
        P->hq = P->hu = nullptr;
        P->stage_bytes = 0;
        if ((st = pim_alloc(P, &P->hq, bytes)) != PIM_OK) return st;
        if ((st = pim_alloc(P, &P->hu, bytes)) != PIM_OK) return st;
        P->stage_bytes = bytes;
    }
    const void* dq = q;
    void* du = u;
    if (hq) {
        PIM_CK(cudaMemcpyAsync(P->hq, q, bytes, cudaMemcpyHostToDevice, s));
        dq = P->hq;
    }
    if (hu) du = P->hu;
    if ((st = apply_run(P, dq, du, nrhs, adj, s)) != PIM_OK) return st;
    if (hu) PIM_CK(cudaMemcpyAsync(u, du, bytes, cudaMemcpyDeviceToHost, s));
    PIM_CK(cudaStreamSynchronize(s));
    return PIM_OK;
}

pim_status pim_apply(pim_plan P, const void* q, void* u, int nrhs, void* stream) {
    return apply_common(P, q, u, nrhs, stream, false);
}

pim_status pim_apply_adjoint(pim_plan P, const void* v, void* w, int nrhs, void* stream) {
    return apply_common(P, v, w, nrhs, stream, true);
}

pim_status pim_position_grad(pim_plan P, const void* q, const void* g, double* grad, int nrhs, void* stream) {
    if (!P || !q || !g || !grad || nrhs < 1) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (!P->pts.box_ptr || !P->with_gradient || !P->pts.dval) {
        pim_set_error("position gradient needs pim_set_points on a plan created with with_gradient = 1");
        return PIM_ERR_STATE;
    }
    return position_grad(P, q, g, grad, nrhs, stream, false);
}

pim_status pim_position_grad_reuse(pim_plan P, const void* q, const void* g, double* grad, void* stream) {
    if (!P || !q || !g || !grad) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (!P->pts.box_ptr || !P->with_gradient || !P->pts.dval) {
        pim_set_error("position gradient needs pim_set_points on a plan created with with_gradient = 1");
        return PIM_ERR_STATE;
    }
    if (P->pot_valid != 3) {
        pim_set_error("no single-RHS forward and adjoint applies on record since the points were last set");
        return PIM_ERR_STATE;
    }
    return position_grad(P, q, g, grad, 1, stream, true);
}

}  // extern "C"

static pim_status position_grad(pim_plan P, const void* q, const void* g, double* grad, int nrhs, void* stream,
                                bool reuse) {
    cudaStream_t s = (cudaStream_t)stream;
    pim_status st;
    if ((st = alloc_grad_buffers(P)) != PIM_OK) return st;
    const size_t bytes = (size_t)P->pts.N * nrhs * data_elem(P);
    const size_t gbytes = (size_t)P->pts.N * 3 * sizeof(double);
    const bool hq = !is_device_ptr(q), hg = !is_device_ptr(g), hd = !is_device_ptr(grad);
    void *dq = (void*)q, *dg = (void*)g;
    double* dgr = grad;
    void *tq = nullptr, *tg = nullptr, *tgr = nullptr;
    if (hq) {
        if ((st = pim_alloc(P, &tq, bytes)) != PIM_OK) return st;
        PIM_CK(cudaMemcpyAsync(tq, q, bytes, cudaMemcpyHostToDevice, s));
        dq = tq;
    }
    if (hg) {
        if ((st = pim_alloc(P, &tg, bytes)) != PIM_OK) return st;
        PIM_CK(cudaMemcpyAsync(tg, g, bytes, cudaMemcpyHostToDevice, s));
        dg = tg;
    }
    if (hd) {
        if ((st = pim_alloc(P, &tgr, gbytes)) != PIM_OK) return st;
        dgr = (double*)tgr;
    }
    st = grad_run(P, dq, dg, dgr, nrhs, s, reuse);
    if (st == PIM_OK && hd) PIM_CK(cudaMemcpyAsync(grad, dgr, gbytes, cudaMemcpyDeviceToHost, s));
    if (hq || hg || hd) PIM_CK(cudaStreamSynchronize(s));
    pim_free(P, tq, bytes);
    pim_free(P, tg, bytes);
    pim_free(P, tgr, gbytes);
    return st;
}

extern "C" {

pim_status pim_update_positions(pim_plan P, const double* xyz) {
    if (!P || (P->pts.N > 0 && !xyz)) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (!P->pts.box_ptr) {
        pim_set_error("update before pim_set_points");
        return PIM_ERR_STATE;
    }
    const int64_t N = P->pts.N;
    PIM_CK(cudaDeviceSynchronize());
    const double* dx = xyz;
    double* tmp = nullptr;
    pim_status st;
    if (N > 0 && !is_device_ptr(xyz)) {
        if ((st = pim_alloc(P, (void**)&tmp, 3 * N * sizeof(double))) != PIM_OK) return st;
        PIM_CK(cudaMemcpy(tmp, xyz, 3 * N * sizeof(double), cudaMemcpyHostToDevice));
        dx = tmp;
    }
    P->pot_valid = 0;
    st = points_update(P, dx, 0);
    pim_free(P, tmp, 3 * N * sizeof(double));
    return st;
}

pim_status pim_last_device_status(pim_plan P) {
    if (!P) return PIM_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        pim_set_error(cudaGetErrorString(cudaGetLastError()));
        return PIM_ERR_CUDA;
    }
    int h = 0;
    PIM_CK(cudaMemcpy(&h, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost));
    PIM_CK(cudaMemset(P->dstatus, 0, sizeof(int)));
    if (h & PIM_DEV_NOT_NEUTRAL) return PIM_ERR_NOT_NEUTRAL;
    if (h & PIM_DEV_TIMEOUT) {
        pim_set_error("a bounded wait of the tensor-core kernel ran out");
        return PIM_ERR_TIMEOUT;
    }
    if (h) return PIM_ERR_DEVICE;
    return PIM_OK;
}

pim_status pim_plan_info(pim_plan P, pim_info* info) {
    if (!P || !info) return PIM_ERR_ARG;
    std::memset(info, 0, sizeof(*info));
    for (int d = 0; d < 3; ++d) {
        info->n[d] = P->n[d];
        info->nf[d] = P->has_far ? P->nf[d] : 0;
    }
    info->p = P->p;
    info->pf = P->pf;
    info->corr_radius = P->b;
    info->precision = P->prec;
    info->corr_mode = P->corr_mode;
    info->periodic_mask = (int)P->pmask;
    info->near_layers = P->layers;
    info->N = P->pts.N;
    info->nnz = P->pts.nnz;
    info->device_bytes = P->bytes;
    info->plan_ms = P->plan_ms;
    info->points_ms = P->points_ms;
    info->launches = P->launches;
    info->gather_variant = P->gather_variant;
    info->gather_variants = gather_variant_count(P);
    info->lf_boxes = P->pts.nlf;
    info->lf_points = P->pts.lf_points;
    info->lf_pairs = P->pts.lf_pairs;
    info->lf_tc_boxes = P->pts.ntc;
    return PIM_OK;
}

pim_status pim_set_profiling(pim_plan P, int on) {
    if (!P) return PIM_ERR_ARG;
    PIM_CK(cudaDeviceSynchronize());
    if (on && !P->prof_ev) {
        const int ne = pim_plan_s::PROF_RING * PIM_NUM_STAGES * 2;
        P->prof_ev = new cudaEvent_t[ne];
        for (int i = 0; i < ne; ++i) PIM_CK(cudaEventCreate(&P->prof_ev[i]));
    }
    P->prof_on = on != 0;
    P->prof_next = 0;
    std::memset(P->prof_mask, 0, sizeof(P->prof_mask));
    return PIM_OK;
}

pim_status pim_stage_times(pim_plan P, double* ms, int n, int64_t* count) {
    if (!P || (n > 0 && !ms)) return PIM_ERR_ARG;
    PIM_CK(cudaDeviceSynchronize());
    for (int st = 0; st < n; ++st) ms[st] = 0.0;
    const int used = P->prof_next < pim_plan_s::PROF_RING ? P->prof_next : pim_plan_s::PROF_RING;
    for (int slot = 0; slot < used && P->prof_ev; ++slot)
        for (int st = 0; st < n && st < PIM_NUM_STAGES; ++st) {
            if (!(P->prof_mask[slot] & (1u << st))) continue;
            float t = 0.f;
            PIM_CK(cudaEventElapsedTime(&t, P->prof_ev[(slot * PIM_NUM_STAGES + st) * 2],
                                        P->prof_ev[(slot * PIM_NUM_STAGES + st) * 2 + 1]));
            ms[st] += t;
        }
    if (count) *count = used;
    return PIM_OK;
}

const char* pim_stage_name(int stage) {
    static const char* names[PIM_NUM_STAGES] = {"permute", "spread", "fft", "gather_correct", "far", "apply",
                                                "lf_exact", "lf_grid", "corr_multi", "lf_tc_gemm"};
    return stage >= 0 && stage < PIM_NUM_STAGES ? names[stage] : nullptr;
}

pim_status pim_debug_copy(pim_plan P, int what, void* host, size_t bytes) {
    if (!P || !host) return PIM_ERR_ARG;
    PIM_CK(cudaDeviceSynchronize());
    const size_t ge = grid_elem(P);
    const size_t G = (size_t)P->n[0] * P->n[1] * P->n[2];
    const size_t N = (size_t)P->pts.N;
    const void* src = nullptr;
    size_t need = 0;
    pim_status st;
    switch (what) {
        case 0:
            if (!P->has_far) return PIM_ERR_STATE;
            src = P->ftab;
            need = (size_t)(2 * P->nf[0] - 1) * (2 * P->nf[1] - 1) * (2 * P->nf[2] - 1) * sizeof(double2);
            break;
        case 1:
            if (!P->qs) return PIM_ERR_STATE;
            need = G * ge;
            if ((st = apply_debug_spread(P, P->gB, 0)) != PIM_OK) return st;
            PIM_CK(cudaDeviceSynchronize());
            src = P->gB;
            break;
        case 2: src = P->gA; need = G * ge; break;
        case 3: src = P->pts.perm; need = N * sizeof(int); break;
        case 4: src = P->pts.row_ptr; need = (N + 1) * sizeof(int64_t); break;
        case 5: src = P->pts.col; need = (size_t)P->pts.nnz * sizeof(uint32_t); break;
        case 6: src = P->pts.val; need = (size_t)P->pts.nnz * sizeof(double2); break;
        case 7:
            if (P->corr_mode != PIM_CORR_COMPACT) return PIM_ERR_STATE;
            src = P->pts.nbig;
            need = N * sizeof(int);
            break;
        default: return PIM_ERR_ARG;
    }
    if (bytes < need) {
        pim_set_error("destination too small");
        return PIM_ERR_ARG;
    }
    if (need == 0) return PIM_OK;
    if (!src) return PIM_ERR_STATE;
    PIM_CK(cudaMemcpy(host, src, need, cudaMemcpyDeviceToHost));
    return PIM_OK;
}

}  // extern "C"
