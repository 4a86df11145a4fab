// pim_apply_batched: several plans (point sets) applied as one unit of work,
// captured once into a CUDA graph and replayed with one launch.
#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "pim_internal.cuh"

namespace {

struct BatchKey {
    std::vector<const void*> ptrs;  // plans, then q, then u
    int nrhs, adj;
    bool operator<(const BatchKey& o) const {
        if (nrhs != o.nrhs) return nrhs < o.nrhs;
        if (adj != o.adj) return adj < o.adj;
        return ptrs < o.ptrs;
    }
};

struct BatchGraph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    std::vector<cudaEvent_t> events;
    size_t nodes = 0;
};

std::mutex g_mu;
std::map<BatchKey, BatchGraph> g_cache;
cudaStream_t g_own = nullptr;  // used when the caller passes the legacy default stream

void destroy_graph(BatchGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
    for (cudaEvent_t e : g.events) cudaEventDestroy(e);
    g.exec = nullptr;
    g.graph = nullptr;
    g.events.clear();
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// Drops every cached graph that uses plan P (called by pim_destroy and
// pim_set_points / pim_update_positions, which change what a graph reads).
void batch_forget(pim_plan P) {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end();) {
        if (std::find(it->first.ptrs.begin(), it->first.ptrs.end(), (const void*)P) != it->first.ptrs.end()) {
            destroy_graph(it->second);
            it = g_cache.erase(it);
        } else {
            ++it;
        }
    }
}

extern "C" pim_status pim_apply_batched(int nplans, pim_plan const* plans, const void* const* q, void* const* u,
                                        int nrhs, int adjoint, void* stream) {
    if (nplans < 1 || !plans || !q || !u || nrhs < 1) {
        pim_set_error("invalid argument");
        return PIM_ERR_ARG;
    }
    for (int i = 0; i < nplans; ++i) {
        if (!plans[i] || !q[i] || !u[i]) {
            pim_set_error("null plan or buffer");
            return PIM_ERR_ARG;
        }
        if (!plans[i]->pts.box_ptr) {
            pim_set_error("a plan has no points");
            return PIM_ERR_STATE;
        }
        if (!is_device_ptr(q[i]) || !is_device_ptr(u[i])) {
            pim_set_error("pim_apply_batched takes device pointers only");
            return PIM_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (plans[j] == plans[i]) {
                pim_set_error("a plan appears twice in one batch (its scratch would be shared)");
                return PIM_ERR_ARG;
            }
    }
    cudaStream_t cs = (cudaStream_t)stream;
    bool own = false;
    if (!cs) {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_own && cudaStreamCreateWithFlags(&g_own, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            pim_set_error("stream creation failed");
            return PIM_ERR_CUDA;
        }
        cs = g_own;
        own = true;
    }
    BatchKey key;
    key.nrhs = nrhs;
    key.adj = adjoint ? 1 : 0;
    for (int i = 0; i < nplans; ++i) key.ptrs.push_back(plans[i]);
    for (int i = 0; i < nplans; ++i) key.ptrs.push_back(q[i]);
    for (int i = 0; i < nplans; ++i) key.ptrs.push_back(u[i]);
    std::unique_lock<std::mutex> lk(g_mu);
    auto it = g_cache.find(key);
    if (it == g_cache.end()) {
        lk.unlock();
        BatchGraph bg;
        pim_status st;
        // each plan runs on its own stream; buffers that an apply would
        // allocate on first use are allocated here, before the capture
        for (int i = 0; i < nplans; ++i)
            if ((st = apply_prepare(plans[i], nrhs, adjoint != 0)) != PIM_OK) return st;
        cudaEvent_t fork;
        PIM_CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
        bg.events.push_back(fork);
        std::vector<cudaEvent_t> done(nplans);
        for (int i = 0; i < nplans; ++i) {
            PIM_CK(cudaEventCreateWithFlags(&done[i], cudaEventDisableTiming));
            bg.events.push_back(done[i]);
        }
        PIM_CK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
        st = PIM_OK;
        if (cudaEventRecord(fork, cs) != cudaSuccess) st = PIM_ERR_CUDA;
        for (int i = 0; i < nplans && st == PIM_OK; ++i) {
            pim_plan P = plans[i];
            if (cudaStreamWaitEvent(P->s_main, fork, 0) != cudaSuccess) st = PIM_ERR_CUDA;
            if (st == PIM_OK) st = apply_run(P, q[i], u[i], nrhs, adjoint != 0, P->s_main);
            if (st == PIM_OK && cudaEventRecord(done[i], P->s_main) != cudaSuccess) st = PIM_ERR_CUDA;
            if (st == PIM_OK && cudaStreamWaitEvent(cs, done[i], 0) != cudaSuccess) st = PIM_ERR_CUDA;
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cs, &graph);
        if (st != PIM_OK || ec != cudaSuccess) {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            destroy_graph(bg);
            pim_set_error("graph capture of the batched apply failed");
            return st != PIM_OK ? st : PIM_ERR_CUDA;
        }
        bg.graph = graph;
        PIM_CK(cudaGraphInstantiate(&bg.exec, graph, 0));
        PIM_CK(cudaGraphGetNodes(graph, nullptr, &bg.nodes));
        lk.lock();
        it = g_cache.emplace(key, bg).first;
    }
    cudaGraphExec_t exec = it->second.exec;
    lk.unlock();
    PIM_CK(cudaGraphLaunch(exec, cs));
    if (own) PIM_CK(cudaStreamSynchronize(cs));
    return PIM_OK;
}
