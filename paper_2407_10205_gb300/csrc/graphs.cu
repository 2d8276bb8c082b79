// graphs.cu -- replay of per-iteration step launches through instantiated CUDA graphs.
// A path whose step kernels read their iteration from device memory (IterCtl) launches
// the same kernel with the same arguments every iteration; a chain of such launches is
// built once as a graph (explicit kernel nodes, no stream capture, so any stream works,
// the legacy default stream included) and replayed, which takes the per-launch host
// cost off the loop.
#include <cstring>
#include <vector>

#include "phia_internal.h"

namespace phia {

namespace {
constexpr int64_t kGraphLen = 100;   // launches per graph
constexpr size_t kMaxGraphs = 4;     // cached graphs per owner (oldest evicted)
}  // namespace

struct StepGraph {
    std::vector<uint8_t> key;
    cudaGraphExec_t exec = nullptr;
};

struct StepGraphCache {
    std::vector<StepGraph> entries;
    std::vector<std::vector<uint8_t>> seen;   // keys met once (a short run builds no graph)
    ~StepGraphCache() {
        for (auto &e : entries)
            if (e.exec) cudaGraphExecDestroy(e.exec);
    }
};

StepGraphCache *step_graphs_new() { return new StepGraphCache(); }
void step_graphs_free(StepGraphCache *c) { delete c; }

namespace {

std::vector<uint8_t> make_key(const void *func, dim3 grid, dim3 block, size_t smem, int64_t len, const void *key,
                              size_t key_bytes, unsigned cluster) {
    std::vector<uint8_t> k(sizeof(func) + 7 * sizeof(unsigned) + sizeof(smem) + sizeof(len) + key_bytes);
    uint8_t *p = k.data();
    const unsigned dims[7] = {grid.x, grid.y, grid.z, block.x, block.y, block.z, cluster};
    memcpy(p, &func, sizeof(func)); p += sizeof(func);
    memcpy(p, dims, sizeof(dims)); p += sizeof(dims);
    memcpy(p, &smem, sizeof(smem)); p += sizeof(smem);
    memcpy(p, &len, sizeof(len)); p += sizeof(len);
    memcpy(p, key, key_bytes);
    return k;
}

cudaError_t build(const void *func, dim3 grid, dim3 block, size_t smem, void **args, int64_t len, unsigned cluster,
                  cudaGraphExec_t *out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    cudaKernelNodeParams kp{};
    kp.func = const_cast<void *>(func);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = args;
    kp.extra = nullptr;
    cudaGraphNode_t prev = nullptr;
    for (int64_t i = 0; i < len && e == cudaSuccess; ++i) {
        cudaGraphNode_t node;
        e = cudaGraphAddKernelNode(&node, g, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
        if (e == cudaSuccess && cluster > 1) {
            cudaKernelNodeAttrValue v{};
            v.clusterDim.x = cluster;
            v.clusterDim.y = 1;
            v.clusterDim.z = 1;
            e = cudaGraphKernelNodeSetAttribute(node, cudaKernelNodeAttributeClusterDimension, &v);
        }
        prev = node;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

cudaError_t launch_one(const void *func, dim3 grid, dim3 block, size_t smem, void **args, unsigned cluster,
                       cudaStream_t st) {
    if (cluster <= 1) return cudaLaunchKernel(func, grid, block, args, smem, st);
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelExC(&cfg, func, args);
}

cudaError_t launch_steps(StepGraphCache *cache, const void *func, dim3 grid, dim3 block, size_t smem, void **args,
                         const void *key, size_t key_bytes, int64_t steps, cudaStream_t st, unsigned cluster) {
    int64_t done = 0;
    if (cache && steps >= 2) {
        const int64_t len = steps < kGraphLen ? steps : kGraphLen;
        const std::vector<uint8_t> k = make_key(func, grid, block, smem, len, key, key_bytes, cluster);
        cudaGraphExec_t exec = nullptr;
        for (auto &e : cache->entries)
            if (e.key == k) exec = e.exec;
        bool build_now = false;
        if (!exec) {
            // Building costs about what a few chunks of direct launches cost: build for a
            // run of several chunks, or on the second run with the same arguments.
            build_now = steps >= 2 * kGraphLen;
            for (auto &sk : cache->seen)
                if (sk == k) build_now = true;
            if (!build_now) {
                if (cache->seen.size() >= 8) cache->seen.erase(cache->seen.begin());
                cache->seen.push_back(k);
            }
        }
        if (build_now) {
            cudaError_t e = build(func, grid, block, smem, args, len, cluster, &exec);
            if (e != cudaSuccess) return e;
            if (cache->entries.size() >= kMaxGraphs) {
                cudaGraphExecDestroy(cache->entries.front().exec);
                cache->entries.erase(cache->entries.begin());
            }
            cache->entries.push_back(StepGraph{k, exec});
        }
        for (; exec && done + len <= steps; done += len) {
            cudaError_t e = cudaGraphLaunch(exec, st);
            if (e != cudaSuccess) return e;
        }
    }
    for (; done < steps; ++done) {
        cudaError_t e = launch_one(func, grid, block, smem, args, cluster, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace phia
