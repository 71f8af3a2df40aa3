// FP32-mixed instantiation of the persistent GFMC engine: FP32 recursion
// vectors and stencil, FP32 warp sums of the Gram products, FP64 above.
#include "gfmc_engine.cuh"

namespace gfmc {

template <int NV>
static cudaError_t launch_nv_f32(const Params& p, cudaStream_t s)
{
    const int smem = engine_smem_bytes(p.K);
    cudaError_t e = cudaFuncSetAttribute(gfmc_engine<float, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    Params q = p;
    void* args[] = {(void*)&q};
    return cudaLaunchCooperativeKernel((void*)gfmc_engine<float, NV>, dim3(p.ncta), dim3(kThreads), args,
                                       (size_t)smem, s);
}

cudaError_t launch_engine_f32(const Params& p, cudaStream_t s) { return launch_nv_f32<kVec>(p, s); }

cudaError_t launch_engine_f32(const Params& p, int nv, cudaStream_t s)
{
    return nv == 2 ? launch_nv_f32<2>(p, s) : launch_nv_f32<kVec>(p, s);
}

cudaError_t engine_max_ctas_f32(int K, int* out)
{
    const int smem = engine_smem_bytes(K);
    cudaError_t e = cudaFuncSetAttribute(gfmc_engine<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gfmc_engine<float>, kThreads, smem);
    if (e != cudaSuccess) return e;
    *out = per_sm;
    return cudaSuccess;
}

}  // namespace gfmc

namespace gfmc {

cudaError_t launch_team_f32(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(gfmc_team_engine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&d_jobs, (void*)&njobs, (void*)&vec_bytes};
    return cudaLaunchCooperativeKernel((void*)gfmc_team_engine<float>, dim3(grid), dim3(kThreads), args, (size_t)smem, s);
}

// The same launch through cudaLaunchKernelEx with the cooperative attribute,
// the form a CUDA graph captures as a cooperative kernel node.
cudaError_t launch_team_ex_f32(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = cudaFuncSetAttribute(gfmc_team_engine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gfmc_team_engine<float>, d_jobs, njobs, vec_bytes);
}

cudaError_t team_max_ctas_f32(int smem, int* out)
{
    cudaError_t e = cudaFuncSetAttribute(gfmc_team_engine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, gfmc_team_engine<float>, kThreads, smem);
}

}  // namespace gfmc

namespace gfmc {

static cudaError_t cluster_config_f32(int C, int smem)
{
    cudaError_t e = cudaFuncSetAttribute(gfmc_cluster_engine<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(gfmc_cluster_engine<float>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaError_t launch_cluster_f32(const TeamJob* d_jobs, int njobs, int C, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = cluster_config_f32(C, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * njobs));
    cfg.blockDim = dim3(cluster_threads<float>());
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gfmc_cluster_engine<float>, d_jobs, vec_bytes);
}

cudaError_t cluster_static_smem_f32(int* out)
{
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, gfmc_cluster_engine<float>);
    if (e == cudaSuccess) *out = (int)a.sharedSizeBytes;
    return e;
}

cudaError_t cluster_max_active_f32(int C, int smem, int* out)
{
    cudaError_t e = cluster_config_f32(C, smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(cluster_threads<float>());
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, gfmc_cluster_engine<float>, &cfg);
}

}  // namespace gfmc
