// Launch of the FP32-mixed single-chain engine on seven thread-block
// clusters (one per local unit vector; gfmc_vcluster.cuh).
#include "gfmc_vcluster.cuh"

namespace gfmc {

namespace {
int vc_smem(int K) { return kVcFixedSmem + K * (int)sizeof(double2); }

cudaError_t vc_config()
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_vc_engine);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(gfmc_vc_engine, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaLaunchConfig_t vc_launch_config(int K, cudaStream_t s, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(kVcClusters * kVcC));
    cfg.blockDim = dim3(kVcNT);
    cfg.dynamicSmemBytes = (size_t)vc_smem(K);
    cfg.stream = s;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)kVcC;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}
}  // namespace

cudaError_t launch_vcluster_f32(const Params& p, cudaStream_t s)
{
    if (p.L != kVcL) return cudaErrorInvalidValue;
    cudaError_t e = vc_config();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = vc_launch_config(p.K, s, attr);
    return cudaLaunchKernelEx(&cfg, gfmc_vc_engine, p);
}

cudaError_t vcluster_max_clusters(int K, int* out)
{
    cudaError_t e = vc_config();
    if (e != cudaSuccess) return e;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = vc_launch_config(K, nullptr, attr);
    return cudaOccupancyMaxActiveClusters(out, gfmc_vc_engine, &cfg);
}

}  // namespace gfmc
