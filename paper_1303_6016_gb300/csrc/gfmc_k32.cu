// FP32-mixed instantiations of the GFMC engines: FP32 recursion vectors and
// stencil, Gram dot products summed in FP32 within a warp (plain, or
// compensated when comp is set) and in FP64 above.
#include "gfmc_engine.cuh"

namespace gfmc {

template <int NV, bool COMP>
static cudaError_t launch_nv_f32(const Params& p, cudaStream_t s)
{
    const int smem = engine_smem_bytes(p.K);
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_engine<float, NV, COMP>);
    if (e != cudaSuccess) return e;
    Params q = p;
    void* args[] = {(void*)&q};
    return cudaLaunchCooperativeKernel((void*)gfmc_engine<float, NV, COMP>, dim3(p.ncta), dim3(kThreads), args,
                                       (size_t)smem, s);
}

cudaError_t launch_engine_f32(const Params& p, cudaStream_t s) { return launch_engine_f32(p, kVec, s); }

cudaError_t launch_engine_f32(const Params& p, int nv, cudaStream_t s)
{
    if (p.comp) return nv == 2 ? launch_nv_f32<2, true>(p, s) : launch_nv_f32<kVec, true>(p, s);
    return nv == 2 ? launch_nv_f32<2, false>(p, s) : launch_nv_f32<kVec, false>(p, s);
}

template <bool COMP>
static cudaError_t max_ctas_f32(int K, int* out)
{
    const int smem = engine_smem_bytes(K);
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_engine<float, kVec, COMP>);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gfmc_engine<float, kVec, COMP>, kThreads, smem);
    if (e != cudaSuccess) return e;
    *out = per_sm;
    return cudaSuccess;
}

cudaError_t engine_max_ctas_f32(int K, int* out)
{
    int a = 0, b = 0;
    cudaError_t e = max_ctas_f32<false>(K, &a);
    if (e == cudaSuccess) e = max_ctas_f32<true>(K, &b);
    if (e == cudaSuccess) *out = a < b ? a : b;
    return e;
}

template <bool COMP>
static cudaError_t team_launch(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s,
                               bool ex)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_team_engine<float, COMP>);
    if (e != cudaSuccess) return e;
    if (!ex) {
        void* args[] = {(void*)&d_jobs, (void*)&njobs, (void*)&vec_bytes};
        return cudaLaunchCooperativeKernel((void*)gfmc_team_engine<float, COMP>, dim3(grid), dim3(kThreads), args,
                                           (size_t)smem, s);
    }
    // the same launch through cudaLaunchKernelEx with the cooperative attribute,
    // the form a CUDA graph captures as a cooperative kernel node
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
    return cudaLaunchKernelEx(&cfg, gfmc_team_engine<float, COMP>, d_jobs, njobs, vec_bytes);
}

cudaError_t launch_team_f32(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s,
                            bool comp)
{
    return comp ? team_launch<true>(d_jobs, njobs, grid, vec_bytes, smem, s, false)
                : team_launch<false>(d_jobs, njobs, grid, vec_bytes, smem, s, false);
}

cudaError_t launch_team_ex_f32(const TeamJob* d_jobs, int njobs, int grid, int vec_bytes, int smem, cudaStream_t s,
                               bool comp)
{
    return comp ? team_launch<true>(d_jobs, njobs, grid, vec_bytes, smem, s, true)
                : team_launch<false>(d_jobs, njobs, grid, vec_bytes, smem, s, true);
}

template <bool COMP>
static cudaError_t team_occupancy(int smem, int* out)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_team_engine<float, COMP>);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(out, gfmc_team_engine<float, COMP>, kThreads, smem);
}

cudaError_t team_max_ctas_f32(int smem, int* out)
{
    int a = 0, b = 0;
    cudaError_t e = team_occupancy<false>(smem, &a);
    if (e == cudaSuccess) e = team_occupancy<true>(smem, &b);
    if (e == cudaSuccess) *out = a < b ? a : b;
    return e;
}

template <bool COMP>
static cudaError_t cluster_config_f32(int C)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_cluster_engine<float, COMP>);
    if (e == cudaSuccess && C > 8)
        e = cudaFuncSetAttribute(gfmc_cluster_engine<float, COMP>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <bool COMP>
static cudaLaunchConfig_t cluster_cfg(int C, int njobs, int smem, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(C * njobs));
    cfg.blockDim = dim3(cluster_threads<float, COMP>());
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

template <bool COMP>
static cudaError_t cluster_launch(const TeamJob* d_jobs, int njobs, int C, int vec_bytes, int smem, cudaStream_t s)
{
    cudaError_t e = cluster_config_f32<COMP>(C);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_cfg<COMP>(C, njobs, smem, s, attr);
    return cudaLaunchKernelEx(&cfg, gfmc_cluster_engine<float, COMP>, d_jobs, vec_bytes);
}

cudaError_t launch_cluster_f32(const TeamJob* d_jobs, int njobs, int C, int vec_bytes, int smem, cudaStream_t s,
                               bool comp)
{
    return comp ? cluster_launch<true>(d_jobs, njobs, C, vec_bytes, smem, s)
                : cluster_launch<false>(d_jobs, njobs, C, vec_bytes, smem, s);
}

cudaError_t cluster_static_smem_f32(int* out)
{
    // the larger of the plain and compensated variants, so one fit check covers both
    cudaFuncAttributes a, b;
    cudaError_t e = cudaFuncGetAttributes(&a, gfmc_cluster_engine<float, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&b, gfmc_cluster_engine<float, true>);
    if (e == cudaSuccess) *out = (int)(a.sharedSizeBytes > b.sharedSizeBytes ? a.sharedSizeBytes : b.sharedSizeBytes);
    return e;
}

template <bool COMP>
static cudaError_t cluster_active(int C, int smem, int* out)
{
    cudaError_t e = cluster_config_f32<COMP>(C);
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_cfg<COMP>(C, 1, smem, nullptr, attr);
    return cudaOccupancyMaxActiveClusters(out, gfmc_cluster_engine<float, COMP>, &cfg);
}

cudaError_t cluster_max_active_f32(int C, int smem, int* out)
{
    int a = 0, b = 0;
    cudaError_t e = cluster_active<false>(C, smem, &a);
    if (e == cudaSuccess) e = cluster_active<true>(C, smem, &b);
    if (e == cudaSuccess) *out = a < b ? a : b;
    return e;
}

}  // namespace gfmc
