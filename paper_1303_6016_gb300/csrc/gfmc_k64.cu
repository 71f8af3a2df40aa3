// FP64 instantiation of the persistent GFMC engine.
#include "gfmc_engine.cuh"

namespace gfmc {

cudaError_t launch_engine_f64(const Params& p, cudaStream_t s)
{
    const int smem = engine_smem_bytes(p.M);
    cudaError_t e = cudaFuncSetAttribute(gfmc_engine<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    Params q = p;
    void* args[] = {(void*)&q};
    return cudaLaunchCooperativeKernel((void*)gfmc_engine<double>, dim3(p.ncta), dim3(kThreads), args,
                                       (size_t)smem, s);
}

cudaError_t engine_max_ctas_f64(int M, int* out)
{
    const int smem = engine_smem_bytes(M);
    cudaError_t e = cudaFuncSetAttribute(gfmc_engine<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gfmc_engine<double>, kThreads, smem);
    if (e != cudaSuccess) return e;
    *out = per_sm;
    return cudaSuccess;
}

}  // namespace gfmc
