// Kernel launches that can be redirected into a CUDA graph under construction.
//
// Every kernel launch of the solvers and operators goes through wd_launch.
// Normally it launches on the given stream.  While the calling thread has a
// GraphSink installed (graph_sink() != nullptr), the launch is instead
// appended to the sink's graph as a kernel node depending on the previous one.
// Graphs are thus built explicitly, without stream capture, so that building
// one never interferes with other threads' work (stream capture forbids, for
// example, a device-wide synchronisation by any thread while it is in
// progress).
//
// Both kinds of launch use programmatic dependent launch (sm_90 and later):
// the kernel may be dispatched once every block of the kernel before it has
// started, instead of after that kernel has ended, so the launch latency and
// the block dispatch overlap the predecessor's last wave.  Every kernel
// launched here therefore begins with grid_dependency_enter(), which waits
// for the predecessor to complete with its writes visible before the kernel
// touches memory.  WD_PDL=0 in the environment turns the overlap off (plain
// serialised launches; the kernels' waits then return at once).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstddef>
#include <cstdlib>
#include <tuple>
#include <type_traits>
#include <utility>

namespace wd {

// Whether wd_launch uses programmatic dependent launch (read once).
inline bool pdl_enabled()
{
    static const bool on = [] {
        const char *v = std::getenv("WD_PDL");
        return !(v && v[0] == '0' && v[1] == 0);
    }();
    return on;
}

struct GraphSink {
    cudaGraph_t graph = nullptr;
    cudaGraphNode_t last = nullptr;
    cudaError_t err = cudaSuccess;
};

// The calling thread's sink (nullptr: launch normally).  Defined in api.cu.
GraphSink *&graph_sink();

namespace launch_detail {
template <typename Tuple, size_t... I>
void fill(Tuple &t, void **params, std::index_sequence<I...>)
{
    ((params[I] = (void *)&std::get<I>(t)), ...);
}
} // namespace launch_detail

template <typename... KArgs, typename... Args>
cudaError_t wd_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args)
{
    GraphSink *g = graph_sink();
    if (!g) {
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        at[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = smem;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = pdl_enabled() ? 1 : 0;
        return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
    }
    std::tuple<std::decay_t<KArgs>...> vals(std::forward<Args>(args)...);
    void *params[sizeof...(KArgs) > 0 ? sizeof...(KArgs) : 1];
    launch_detail::fill(vals, params, std::index_sequence_for<KArgs...>{});
    cudaKernelNodeParams p{};
    p.func = (void *)kernel;
    p.gridDim = grid;
    p.blockDim = block;
    p.sharedMemBytes = (unsigned)smem;
    p.kernelParams = params;
    p.extra = nullptr;
    // a sink holds kernel nodes only, so every edge joins two kernels and may
    // be programmatic
    cudaGraphEdgeData ed = {};
    if (pdl_enabled()) {
        ed.from_port = cudaGraphKernelNodePortProgrammatic;
        ed.type = cudaGraphDependencyTypeProgrammatic;
    }
    cudaGraphNode_t node;
    cudaError_t e = cudaGraphAddKernelNode(&node, g->graph, nullptr, 0, &p);
    if (e == cudaSuccess && g->last) e = cudaGraphAddDependencies(g->graph, &g->last, &node, &ed, 1);
    if (e == cudaSuccess) g->last = node;
    else if (g->err == cudaSuccess) g->err = e;
    return e;
}

// SM clock of device `dev` (-1: the current one) in kHz, queried once per
// device: the query takes hundreds of microseconds, far longer than a launch.
// Used to turn the bounded waits' limits from seconds into clock cycles.
inline int device_clock_khz(int dev = -1)
{
    static std::atomic<int> cache[64] = {};
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return 2000000;
    if (dev < 0 || dev >= 64) return 2000000;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v == 0) {
        if (cudaDeviceGetAttribute(&v, cudaDevAttrClockRate, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 2000000;
        }
        cache[dev].store(v, std::memory_order_relaxed);
    }
    return v;
}

} // namespace wd
