// CUDA-graph replay of the phases of the batched determinant. Each phase
// runs persistent kernels (one CTA or cluster per job) over job arrays in
// device memory, so its launch sequence depends only on the shape of the
// batch (job counts and size bounds), not on the data: the job arrays are
// copied into a fixed device buffer, and the sequence is captured once per
// shape and replayed. A shape seen for the first time runs eagerly (which
// also sets the kernels' attributes outside any capture); the second time
// it is captured (thread-local capture mode) and instantiated; later calls
// only upload their jobs and launch the graph.
//
// State is per host thread (the serving workers each have their own), so a
// graph is never replayed concurrently with itself and the fixed buffer is
// never overwritten while a replay that reads it is in flight: every batched
// call synchronises its stream before it returns. Graphs are captured and
// replayed on a private stream of the thread (the caller's stream may be the
// legacy default stream, which cannot be captured), ordered after the
// caller's stream by an event and before its later work by another.
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "idet_internal.cuh"

namespace idet {

namespace {

struct GraphState {
    void *buf = nullptr;
    size_t cap = 0;
    int device = -1;
    cudaStream_t ps = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    std::unordered_map<uint64_t, std::pair<cudaGraphExec_t, unsigned>> execs;
    std::unordered_set<uint64_t> seen;
    std::vector<unsigned char> host;
    void clear() {
        for (auto &kv : execs) cudaGraphExecDestroy(kv.second.first);
        execs.clear();
        seen.clear();
    }
    void release() {
        clear();
        if (buf) cudaFree(buf);
        if (ps) cudaStreamDestroy(ps);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        buf = nullptr;
        cap = 0;
        ps = nullptr;
        ev_in = ev_out = nullptr;
    }
    ~GraphState() { release(); }
};

thread_local GraphState t_gs;

uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

}  // namespace

int run_phase_graph(cudaStream_t s, uint64_t key, const std::vector<JobBlob> &blobs,
                    const std::function<int(const std::vector<const void *> &, cudaStream_t)> &record) {
    GraphState &G = t_gs;
    int dev = 0;
    IDET_CUDA_TRY(cudaGetDevice(&dev));
    if (dev != G.device) {
        G.release();
        G.device = dev;
    }
    if (!G.ps) {
        IDET_CUDA_TRY(cudaStreamCreateWithFlags(&G.ps, cudaStreamNonBlocking));
        IDET_CUDA_TRY(cudaEventCreateWithFlags(&G.ev_in, cudaEventDisableTiming));
        IDET_CUDA_TRY(cudaEventCreateWithFlags(&G.ev_out, cudaEventDisableTiming));
    }
    // lay the blobs out at 256-byte offsets; the layout is part of the key
    std::vector<size_t> off(blobs.size());
    size_t total = 0;
    for (size_t i = 0; i < blobs.size(); ++i) {
        off[i] = total;
        total += (blobs[i].bytes + 255) / 256 * 256;
        key = mix(key, blobs[i].bytes);
    }
    if (total > G.cap) {
        // the old buffer may still be read by this thread's last replay
        IDET_CUDA_TRY(cudaStreamSynchronize(s));
        G.clear();
        if (G.buf) cudaFree(G.buf);
        G.buf = nullptr;
        const size_t cap = std::max<size_t>(total * 2, (size_t)1 << 20);
        IDET_CUDA_TRY(cudaMalloc(&G.buf, cap));
        G.cap = cap;
    }
    G.host.assign(total, 0);
    for (size_t i = 0; i < blobs.size(); ++i)
        if (blobs[i].bytes) memcpy(G.host.data() + off[i], blobs[i].data, blobs[i].bytes);
    if (total)
        IDET_CUDA_TRY(cudaMemcpyAsync(G.buf, G.host.data(), total, cudaMemcpyHostToDevice, s));
    std::vector<const void *> dev_ptrs(blobs.size());
    for (size_t i = 0; i < blobs.size(); ++i) dev_ptrs[i] = (const unsigned char *)G.buf + off[i];
    auto replay = [&](cudaGraphExec_t exec, unsigned nk) -> int {
        IDET_CUDA_TRY(cudaEventRecord(G.ev_in, s));
        IDET_CUDA_TRY(cudaStreamWaitEvent(G.ps, G.ev_in, 0));
        IDET_CUDA_TRY(cudaGraphLaunch(exec, G.ps));
        IDET_CUDA_TRY(cudaEventRecord(G.ev_out, G.ps));
        IDET_CUDA_TRY(cudaStreamWaitEvent(s, G.ev_out, 0));
        count_launch(nk);
        return IDET_OK;
    };
    auto hit = G.execs.find(key);
    if (hit != G.execs.end()) return replay(hit->second.first, hit->second.second);
    if (!G.seen.count(key)) {  // first time: run eagerly
        G.seen.insert(key);
        return record(dev_ptrs, s);
    }
    cudaGraph_t graph = nullptr;
    IDET_CUDA_TRY(cudaStreamBeginCapture(G.ps, cudaStreamCaptureModeThreadLocal));
    const unsigned long long l0 = g_launches.load();
    const int rc = record(dev_ptrs, G.ps);
    const unsigned nk = (unsigned)(g_launches.load() - l0);
    g_launches.fetch_sub(nk);  // captured, not launched
    const cudaError_t ec = cudaStreamEndCapture(G.ps, &graph);
    if (rc != IDET_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (ec != cudaSuccess) {
        cudaGetLastError();
        set_last_error("batched phase capture: %s", cudaGetErrorString(ec));
        return IDET_ERR_CUDA;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        set_last_error("batched phase graph: %s", cudaGetErrorString(ei));
        return IDET_ERR_CUDA;
    }
    G.execs[key] = {exec, nk};
    return replay(exec, nk);
}

}  // namespace idet
