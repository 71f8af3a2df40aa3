// FP64 instantiation of the persistent GFMC engine.
#include "gfmc_engine.cuh"

namespace gfmc {

template <int NV, bool SPLIT = false>
static cudaError_t launch_nv_f64(const Params& p, cudaStream_t s)
{
    const int smem = single_smem_bytes(p.K, 0, p.prefetch ? p.win_max : 0);
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_engine<double, NV, false, SPLIT>);
    if (e != cudaSuccess) return e;
    Params q = p;
    void* args[] = {(void*)&q};
    return cudaLaunchCooperativeKernel((void*)gfmc_engine<double, NV, false, SPLIT>, dim3(p.ncta),
                                       dim3(engine_threads<double, NV>()), args, (size_t)smem, s);
}

// p.bip == 2: the instantiation for tiles of at least 128 sites (halo-only
// prefetch, group sums beside the units)
cudaError_t launch_engine_f64(const Params& p, cudaStream_t s)
{
    return p.bip == 2 ? launch_nv_f64<kVec, true>(p, s) : launch_nv_f64<kVec>(p, s);
}

cudaError_t launch_engine_f64(const Params& p, int nv, cudaStream_t s)
{
    return nv == 2 ? launch_nv_f64<2>(p, s) : launch_engine_f64(p, s);
}

cudaError_t engine_static_smem_f64(int* out)
{
    // the larger of the two 7-vector instantiations, so one fit check covers both
    cudaFuncAttributes a, b;
    cudaError_t e = cudaFuncGetAttributes(&a, gfmc_engine<double, kVec>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&b, gfmc_engine<double, kVec, false, true>);
    if (e == cudaSuccess) *out = (int)(a.sharedSizeBytes > b.sharedSizeBytes ? a.sharedSizeBytes : b.sharedSizeBytes);
    return e;
}

cudaError_t engine_max_ctas_f64(int K, int* out)
{
    const int smem = single_smem_bytes(K, 0);
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_engine<double>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gfmc_engine<double>, engine_threads<double, kVec>(),
                                                      smem);
    if (e != cudaSuccess) return e;
    *out = per_sm;
    return cudaSuccess;
}

}  // namespace gfmc

namespace gfmc {

cudaError_t launch_team_f64(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_team_engine<double>);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&d_jobs, (void*)&njobs, (void*)&vec_bytes};
    return cudaLaunchCooperativeKernel((void*)gfmc_team_engine<double>, dim3(grid), dim3(kThreads), args, (size_t)smem, s);
}

// The same launch through cudaLaunchKernelEx with the cooperative attribute,
// the form a CUDA graph captures as a cooperative kernel node.
cudaError_t launch_team_ex_f64(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_team_engine<double>);
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
    return cudaLaunchKernelEx(&cfg, gfmc_team_engine<double>, d_jobs, njobs, vec_bytes);
}

cudaError_t team_max_ctas_f64(int smem, int* out)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_team_engine<double>);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, gfmc_team_engine<double>, kThreads, smem);
}

}  // namespace gfmc

namespace gfmc {

static cudaError_t cluster_config_f64(int C)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_cluster_engine<double>);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(gfmc_cluster_engine<double>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaError_t launch_cluster_f64(const TeamJob* d_jobs, int njobs, int C, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = cluster_config_f64(C);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * njobs));
    cfg.blockDim = dim3(cluster_threads<double>());
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, gfmc_cluster_engine<double>, d_jobs, vec_bytes);
}

cudaError_t cluster_static_smem_f64(int* out)
{
    cudaFuncAttributes a;
    const cudaError_t e = cudaFuncGetAttributes(&a, gfmc_cluster_engine<double>);
    if (e == cudaSuccess) *out = (int)a.sharedSizeBytes;
    return e;
}

cudaError_t cluster_max_active_f64(int C, int smem, int* out)
{
    cudaError_t e = cluster_config_f64(C);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)C);
    cfg.blockDim = dim3(cluster_threads<double>());
    cfg.dynamicSmemBytes = (size_t)smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(out, gfmc_cluster_engine<double>, &cfg);
}

}  // namespace gfmc
