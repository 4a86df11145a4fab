// pim_apply_noalloc: the apply with its per-call scratch in a fixed device
// array that the library owns for the life of the process, so that the call
// itself allocates nothing.
//
// Who needs it: code that must not allocate device memory at the time it
// applies the operator -- for example a solver step running under a memory
// budget that forbids growth after start-up, a caller that runs while a
// stream-ordered allocator or a graph capture is active on another thread,
// or a host language runtime that can only pass in buffers it already owns.
// The plan's persistent tables (spectra, correction list, stencils) are
// created earlier by pim_plan_create / pim_set_points, when allocation is
// allowed.
#include <mutex>

#include "pim_internal.cuh"

namespace {

// 32 MiB of scratch per GPU that loads the library, held until exit.
constexpr size_t NOALLOC_BYTES = 32ull << 20;
static __device__ __align__(256) unsigned char pim_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
// per device: the address of the array in the context it was looked up in,
// and that context's unique id (0: unknown, look it up again)
void* g_addr[MAX_DEVICES] = {nullptr};
unsigned long long g_ctx[MAX_DEVICES] = {0};

// Unique id of the calling thread's current CUDA context (driver
// cuCtxGetCurrent + cuCtxGetId, found through the runtime's entry-point
// query), or 0 if it cannot be had.  A context that is destroyed and
// created again -- cudaDeviceReset, a harness that resets between cases --
// gets a new id, and its module a new copy of the array.
unsigned long long current_context_id() {
    using get_current_t = int (*)(void**);
    using get_id_t = int (*)(void*, unsigned long long*);
    static get_current_t get_current = nullptr;
    static get_id_t get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        looked = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (get_current_t)f1;
            get_id = (get_id_t)f2;
        }
        cudaGetLastError();
    }
    if (!get_current || !get_id) return 0;
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" pim_status pim_apply_noalloc(pim_plan P, const void* q, void* u, int nrhs, int adjoint, void* stream) {
    if (!P || !q || !u || nrhs < 1) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    if (!P->pts.box_ptr) {
        pim_set_error("apply before pim_set_points");
        return PIM_ERR_STATE;
    }
    if (!is_device_ptr(q) || !is_device_ptr(u)) {
        pim_set_error("pim_apply_noalloc takes device pointers only (host buffers would need staging memory)");
        return PIM_ERR_ARG;
    }
    // set-up once per device and context: the device address of the scratch
    // array in the current context (looked up again if the context changed)
    int dev = 0;
    PIM_CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= MAX_DEVICES) {
        pim_set_error("device index out of range");
        return PIM_ERR_ARG;
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const unsigned long long ctx = current_context_id();
        if (!g_addr[dev] || ctx == 0 || ctx != g_ctx[dev]) {
            void* ptr = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&ptr, pim_noalloc_scratch);
            if (e != cudaSuccess) {
                cudaGetLastError();
                pim_set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
                return PIM_ERR_CUDA;
            }
            g_addr[dev] = ptr;
            g_ctx[dev] = ctx;
        }
        base = g_addr[dev];
    }
    // carve the per-call scratch of the apply out of the array
    const size_t ge = P->prec == PIM_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t N = (size_t)P->pts.N;
    const size_t G = (size_t)P->n[0] * P->n[1] * P->n[2];
    const size_t GB = (size_t)P->n[2] * P->n[1] * P->ng.L[0];
    const size_t GC = (size_t)P->n[2] * P->ng.L[1] * P->ng.L[0];
    const size_t np3 = (size_t)(P->p + 1) * (P->p + 1) * (P->p + 1);
    const size_t mom = (size_t)(P->pts.nd > 0 ? P->pts.nd : 1) * np3 * ge;
    size_t Gf = 0, fB = 0, fC = 0;
    if (P->has_far) {
        Gf = (size_t)P->nf[0] * P->nf[1] * P->nf[2];
        fB = (size_t)P->nf[2] * P->nf[1] * P->fg.L[0];
        fC = (size_t)P->nf[2] * P->fg.L[1] * P->fg.L[0];
    }
    const size_t sizes[11] = {N * ge,  N * ge,  G * ge, GB * ge, GC * ge, mom, (size_t)P->far_chunks * Gf * ge,
                              Gf * sizeof(double2), fB * sizeof(double2), fC * sizeof(double2),
                              P->has_far ? N * ge : 0};
    size_t need = 0;
    for (size_t b : sizes) need += up256(b);
    if (need > NOALLOC_BYTES) {
        pim_set_error("plan needs " + std::to_string(need) + " bytes of scratch; pim_apply_noalloc has " +
                      std::to_string(NOALLOC_BYTES));
        return PIM_ERR_ARG;
    }
    unsigned char* cur = static_cast<unsigned char*>(base);
    void* ptrs[11];
    for (int i = 0; i < 11; ++i) {
        ptrs[i] = sizes[i] ? cur : nullptr;
        cur += up256(sizes[i]);
    }
    // run the apply with the plan's scratch fields pointing into the array
    void* save[11] = {P->qs, P->us, P->gA, P->gB, P->gC, P->pts.mom, P->fpart, P->fA, P->fB, P->fC, P->ufp};
    P->qs = ptrs[0];
    P->us = ptrs[1];
    P->gA = ptrs[2];
    P->gB = ptrs[3];
    P->gC = ptrs[4];
    P->pts.mom = ptrs[5];
    if (P->has_far) {
        P->fpart = ptrs[6];
        P->fA = (double2*)ptrs[7];
        P->fB = (double2*)ptrs[8];
        P->fC = (double2*)ptrs[9];
        P->ufp = ptrs[10];
    }
    const bool no_multi = P->no_multi;
    void* ulf = P->ulf;
    P->no_multi = true;  // the multi-RHS path would allocate its source buffer
    P->keep_off = true;  // the grid potentials live in the borrowed scratch
    P->ulf = nullptr;    // list-free boxes: the exact and grid parts added in turn, no buffer
    const pim_status st = apply_run(P, q, u, nrhs, adjoint != 0, (cudaStream_t)stream);
    P->no_multi = no_multi;
    P->keep_off = false;
    P->ulf = ulf;
    P->qs = save[0];
    P->us = save[1];
    P->gA = save[2];
    P->gB = save[3];
    P->gC = save[4];
    P->pts.mom = save[5];
    P->fpart = save[6];
    P->fA = (double2*)save[7];
    P->fB = (double2*)save[8];
    P->fC = (double2*)save[9];
    P->ufp = save[10];
    return st;
}
