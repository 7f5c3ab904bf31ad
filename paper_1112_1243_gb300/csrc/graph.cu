// CUDA-graph capture of library calls, with the solver loops as device-side
// conditional WHILE nodes.
//
// A hierarchical step (proposal, block filter, stochastic global step) is a
// few thousand kernel launches whose trip counts depend on convergence.  In
// eager mode the host polls solver states every few iterations; inside a
// capture every such loop becomes one conditional node: its body graph holds
// one pass of the loop and ends in a one-thread kernel that sets the node's
// condition from the solver states on the device.  The step then runs with
// no host round trip, and a replay re-runs the same buffers with the random
// streams advanced by a device-resident counter offset.
#include <climits>
#include <cstring>

#include "dd_internal.h"

bool dd_stream_capturing(dd_handle* h) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(h->stream, &cs) != cudaSuccess) return false;
    return cs == cudaStreamCaptureStatusActive;
}

int upload_cached(dd_handle* h, int slot, void* dst, const void* src, size_t bytes) {
    std::vector<char>& c = h->upload_cache[slot];
    const size_t head = sizeof(void*) + sizeof(size_t);
    const bool same = c.size() == head + bytes && std::memcmp(c.data(), &dst, sizeof(void*)) == 0 &&
                      std::memcmp(c.data() + head, src, bytes) == 0;
    if (same) return DD_OK;
    if (dd_stream_capturing(h))
        return dd_fail(h, DD_ERR_UNSUPPORTED,
                       "descriptor tables differ from the last eager call: run the call once outside the capture");
    c.resize(head + bytes);
    std::memcpy(c.data(), &dst, sizeof(void*));
    std::memcpy(c.data() + sizeof(void*), &bytes, sizeof(size_t));
    std::memcpy(c.data() + head, src, bytes);
    DD_CUDA(h, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, h->stream));
    return DD_OK;
}

namespace {

// counters of one loop: [0] passes of the body, [1] running iteration total
__global__ void loop_arm_kernel(cudaGraphConditionalHandle c, int* ctr) {
    ctr[0] = 0;
    ctr[1] = 0;
    cudaGraphSetConditional(c, 1u);
}

__global__ void loop_cond_kernel(cudaGraphConditionalHandle c, LoopCond L, int* ctr, int* status) {
    const int trips = ++ctr[0];
    bool any = false;
    int flags = 0;
    for (int k = 0; k < L.nrhs; ++k) {
        any = any || L.st[k].active;
        flags |= L.st[k].flags;
    }
    if (L.it_src) {
        long long t = ctr[1];
        for (int k = 0; k < L.nrhs; ++k) t += L.it_src[k].iters;
        ctr[1] = (int)(t < INT_MAX ? t : INT_MAX);
        if (t >= L.max_total) any = false;
    }
    if (L.numeric && (flags & 2)) {
        raise_status(status, DD_ERR_NUMERIC);
        any = false;
    }
    cudaGraphSetConditional(c, (any && trips < L.max_trips) ? 1u : 0u);
}

__global__ void set_u64_kernel(unsigned long long* p, unsigned long long v) { *p = v; }

}  // namespace

int dd_loop(dd_handle* h, const std::function<int()>& body, const std::function<int(bool&)>& host_more,
            const LoopCond& cond) {
    if (!dd_stream_capturing(h)) {
        for (;;) {
            int rc = body();
            if (rc) return rc;
            bool more = false;
            rc = host_more(more);
            if (rc) return rc;
            if (!more) return DD_OK;
        }
    }
    const int depth = h->loop_depth;
    if (2 * depth + 2 > DD_LOOP_SLOTS) return dd_fail(h, DD_ERR_UNSUPPORTED, "solver loops nested too deeply");
    int* ctr = h->d_loop + 2 * depth;
    cudaStreamCaptureStatus cs;
    cudaGraph_t g = nullptr;
    DD_CUDA(h, cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, nullptr, nullptr, nullptr));
    cudaGraphConditionalHandle ch;
    DD_CUDA(h, cudaGraphConditionalHandleCreate(&ch, g, 1, cudaGraphCondAssignDefault));
    // the condition is set explicitly before every entry into the loop (a
    // default value would apply once per graph launch, not per entry of a
    // loop nested in another loop's body)
    DD_KLAUNCH(h, loop_arm_kernel<<<1, 1, 0, h->stream>>>(ch, ctr));
    DD_LAUNCH_CHECK(h, "loop_arm_kernel");
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    DD_CUDA(h, cudaStreamGetCaptureInfo(h->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np{};
    std::memset((void*)&np, 0, sizeof(np));
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = ch;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    DD_CUDA(h, cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    cudaGraph_t body_graph = np.conditional.phGraph_out[0];
    DD_CUDA(h, cudaStreamUpdateCaptureDependencies(h->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    while ((int)h->body_streams.size() <= depth) {
        cudaStream_t st;
        DD_CUDA(h, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        h->body_streams.push_back(st);
    }
    cudaStream_t parent = h->stream, side = h->body_streams[depth];
    DD_CUDA(h, cudaStreamBeginCaptureToGraph(side, body_graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    h->stream = side;
    h->loop_depth = depth + 1;
    int rc = body();
    if (!rc) {
        DD_KLAUNCH(h, loop_cond_kernel<<<1, 1, 0, side>>>(ch, cond, ctr, h->d_status));
        if (cudaGetLastError() != cudaSuccess) rc = DD_ERR_CUDA;
    }
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(side, &captured);
    h->stream = parent;
    h->loop_depth = depth;
    if (rc) return rc;
    if (e != cudaSuccess) return dd_cuda_check(h, e, "conditional loop body capture");
    return DD_OK;
}

// ------------------------------------------------------------- entry points
struct dd_graph {
    dd_handle* h = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int dd_graph_begin(dd_t h) {
    int rc = dd_require_ws(h);
    if (rc) return rc;
    if (h->capturing) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_graph_begin: a capture is already open");
    if (!h->cap_stream) DD_CUDA(h, cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    // capture on the handle's private stream, so that the caller's stream
    // may be the legacy default stream (which cannot be captured)
    h->user_stream = h->stream;
    DD_CUDA(h, cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeRelaxed));
    h->stream = h->cap_stream;
    h->capturing = true;
    return DD_OK;
}

extern "C" int dd_graph_end(dd_t h, dd_graph_t* out) {
    if (!h || !out) return DD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!h->capturing) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_graph_end: no open capture");
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap_stream, &graph);
    h->stream = h->user_stream;
    h->capturing = false;
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return dd_cuda_check(h, e, "cudaStreamEndCapture");
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return dd_cuda_check(h, e, "cudaGraphInstantiate");
    }
    dd_graph* g = new dd_graph();
    g->h = h;
    g->graph = graph;
    g->exec = exec;
    *out = g;
    return DD_OK;
}

extern "C" int dd_graph_launch(dd_graph_t g, unsigned long long ctr_offset) {
    if (!g || !g->h) return DD_ERR_INVALID_ARG;
    dd_handle* h = g->h;
    if (h->capturing) return dd_fail(h, DD_ERR_INVALID_ARG, "dd_graph_launch: a capture is open on the handle");
    DD_KLAUNCH(h, set_u64_kernel<<<1, 1, 0, h->stream>>>(h->d_ctr_off, ctr_offset));
    DD_CUDA(h, cudaGraphLaunch(g->exec, h->stream));
    DD_KLAUNCH(h, set_u64_kernel<<<1, 1, 0, h->stream>>>(h->d_ctr_off, 0ull));
    DD_LAUNCH_CHECK(h, "dd_graph_launch");
    return DD_OK;
}

extern "C" int dd_graph_nodes(dd_graph_t g, size_t* nodes) {
    if (!g || !nodes) return DD_ERR_INVALID_ARG;
    size_t n = 0;
    if (cudaGraphGetNodes(g->graph, nullptr, &n) != cudaSuccess) return DD_ERR_CUDA;
    *nodes = n;
    return DD_OK;
}

extern "C" int dd_graph_destroy(dd_graph_t g) {
    if (!g) return DD_ERR_INVALID_ARG;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return DD_OK;
}
