// CUDA-graph replay of the operator and preconditioner applications.  A
// matvec is ~20-30 small launches (P2M, translations per level, near field),
// and the learned preconditioner ~20 more; replaying them as one captured
// graph removes the per-launch host cost and the gaps between kernels.  The
// graph reads and writes two staging vectors owned by the cache (captured
// pointers are fixed); a replay copies the caller's input in, launches the
// graph and copies the result out.  One graph per number of right-hand
// sides; the body runs once uncaptured first so that every lazily built
// buffer or tile list exists before capture.  An owner that reallocates a
// buffer a graph may have captured bumps its generation counter; graphs of
// an older generation are captured again before their next replay.  Capture uses a private
// stream; replays go to the caller's stream.
#include <atomic>
#include <functional>
#include <map>

#include "common.cuh"

struct GraphEntry {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cd* gx = nullptr;
    cd* gy = nullptr;
    long long kernels = 0;
    long long gen = -1;           // owner's buffer generation at capture
};
struct GraphCache {
    std::map<int, GraphEntry> m;
    cudaStream_t cap = nullptr;   // capture stream (the legacy default stream cannot be captured)
};

long long fb_launch_count();

void fb_graph_free(void*& cache) {
    GraphCache* gc = (GraphCache*)cache;
    if (!gc) return;
    for (auto& kv : gc->m) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
        dfree(kv.second.gx);
        dfree(kv.second.gy);
    }
    if (gc->cap) cudaStreamDestroy(gc->cap);
    delete gc;
    cache = nullptr;
}

static void drop_entry(GraphEntry& e) {
    if (e.exec) cudaGraphExecDestroy(e.exec);
    if (e.graph) cudaGraphDestroy(e.graph);
    dfree(e.gx);
    dfree(e.gy);
    e = GraphEntry{};
}

fb_status fb_graph_run(void*& cache, int key, int64_t in_elems, int64_t out_elems, const cd* x, cd* y,
                       cudaStream_t s, const std::function<fb_status(const cd*, cd*, cudaStream_t)>& body,
                       const long long* gen) {
    // inside another object's capture (e.g. a preconditioner whose base
    // applies a graphed operator): run the body directly, it is captured
    // into the enclosing graph
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    FB_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) return body(x, y, s);
    if (!cache) cache = new GraphCache();
    GraphCache* gc = (GraphCache*)cache;
    auto it = gc->m.find(key);
    if (it != gc->m.end() && gen && it->second.gen != *gen) {
        // the owner reallocated buffers the graph captured: capture again
        FB_CUDA(cudaStreamSynchronize(s));
        drop_entry(it->second);
        gc->m.erase(it);
        it = gc->m.end();
    }
    if (it == gc->m.end()) {
        GraphEntry e;
        FB_CHECK(dalloc(&e.gx, in_elems));
        FB_CHECK(dalloc(&e.gy, out_elems));
        FB_CUDA(cudaMemsetAsync(e.gx, 0, sizeof(cd) * in_elems, s));
        FB_CHECK(body(e.gx, e.gy, s));      // builds every lazy buffer outside the capture
        FB_CUDA(cudaStreamSynchronize(s));
        if (!gc->cap) FB_CUDA(cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking));
        long long before = fb_launch_count();
        FB_CUDA(cudaStreamBeginCapture(gc->cap, cudaStreamCaptureModeThreadLocal));
        fb_status st = body(e.gx, e.gy, gc->cap);
        cudaGraph_t g = nullptr;
        cudaError_t ce = cudaStreamEndCapture(gc->cap, &g);
        long long captured = fb_launch_count() - before;
        fb_count_launch(-captured);          // kernels are counted per replay instead
        if (st != FB_OK || ce != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            dfree(e.gx);
            dfree(e.gy);
            if (st != FB_OK) return st;
            return fb_fail(FB_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        }
        e.graph = g;
        e.kernels = captured;
        e.gen = gen ? *gen : 0;   // read after the uncaptured run, which may have grown buffers
        cudaError_t ie = cudaGraphInstantiate(&e.exec, g, 0);
        if (ie != cudaSuccess) {
            cudaGraphDestroy(g);
            dfree(e.gx);
            dfree(e.gy);
            return fb_fail(FB_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
        }
        it = gc->m.emplace(key, e).first;
    }
    GraphEntry& e = it->second;
    FB_CUDA(cudaMemcpyAsync(e.gx, x, sizeof(cd) * in_elems, cudaMemcpyDeviceToDevice, s));
    FB_CUDA(cudaGraphLaunch(e.exec, s));
    FB_CUDA(cudaMemcpyAsync(y, e.gy, sizeof(cd) * out_elems, cudaMemcpyDeviceToDevice, s));
    fb_count_launch(e.kernels);
    return FB_OK;
}
