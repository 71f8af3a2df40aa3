// gfmc_server.cu -- the device-resident request loop of the serving layer.
//
// One persistent cooperative launch whose CTAs are split into slots (teams).
// Each slot runs posted jobs -- "continue chain X by n updates" -- one after
// another, in either precision, while the other slots run theirs: requests
// that arrive while others are on the GPU are admitted as soon as a slot is
// free, and their work overlaps on the device.
//
// Mailbox protocol of a slot (all waits bounded):
//   host    writes the job (copy engine), then the slot's sequence number;
//   CTA 0   of the slot polls the sequence number; on a new one it publishes
//           it in the slot's command word; on shutdown, or once every slot
//           of the launch has been idle for idle_budget cycles, it publishes
//           EXIT;
//   others  poll the command word and follow it, so a slot never splits;
//   slot    runs the job (run_chain, multi-site variant), meets at the job's
//           barrier, and CTA 0 writes the sequence number into the host-mapped
//           done word.
// The launch ends as a whole: a slot idle for idle_budget cycles joins the
// launch's idle count (and leaves it when work arrives); the slot whose entry
// makes every slot idle raises the exit word, which every slot's CTA 0 obeys.
// A slot that exited on its own while others stayed busy would leave its next
// job waiting for the whole launch to end.  A slot idle for kIdleCap budgets
// exits regardless, so every wait stays bounded.  A posted job that the
// kernel did not take before the exit is taken by the next launch (each
// launch starts from the done words).
#include "gfmc_engine.cuh"

namespace gfmc {

constexpr unsigned kExit = 0xFFFFFFFFu;
constexpr long long kIdleCap = 64;  // idle budgets after which a slot exits even if others are busy

__device__ __forceinline__ void st_release_sys_u32(unsigned* a, unsigned v)
{
    asm volatile("st.release.sys.global.u32 [%0], %1;" ::"l"(a), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire_sys_u32(const unsigned* a)
{
    unsigned v;
    asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(a) : "memory");
    return v;
}

__global__ void __launch_bounds__(kThreads, 1) gfmc_server_kernel(ServerArgs a)
{
    extern __shared__ double2 work[];
    __shared__ Params sp;
    __shared__ int s_slot, s_cta, s_prec;
    __shared__ unsigned s_cmd;
    if (threadIdx.x == 0) {
        int j = 0;
        while (j + 1 < a.nslots && a.slots[j + 1].cta0 <= (int)blockIdx.x) ++j;
        s_slot = j;
        s_cta = (int)blockIdx.x - a.slots[j].cta0;
    }
    __syncthreads();
    SlotCtl* sl = a.slots + s_slot;
    unsigned last = ld_acquire_sys_u32(a.done + s_slot);
    for (;;) {
        if (threadIdx.x == 0) {
            unsigned cmd = kExit;
            const long long t0 = clock64();
            if (s_cta == 0) {
                bool idle = false;  // this slot is counted in quiesce[0]
                for (;;) {
                    const unsigned q = ld_acquire_u32(&sl->seq);
                    if (q != last) {
                        if (idle) {
                            if (ld_acquire_u32(a.quiesce + 1) != 0u) break;  // ending: the job goes to the next launch
                            atomicSub(a.quiesce, 1u);
                        }
                        cmd = q;
                        break;
                    }
                    if (ld_acquire_u32(a.shutdown) != 0u || ld_acquire_u32(a.quiesce + 1) != 0u) break;
                    const long long waited = clock64() - t0;
                    if (!idle && waited > a.idle_budget) {
                        idle = true;
                        if (atomicAdd(a.quiesce, 1u) + 1u == (unsigned)a.nslots) st_release_u32(a.quiesce + 1, 1u);
                    }
                    if (waited > kIdleCap * a.idle_budget) break;
                    __nanosleep(500);
                }
                st_release_u32(&sl->cmd, cmd);
            } else {
                for (;;) {
                    const unsigned c = ld_acquire_u32(&sl->cmd);
                    if (c != last) {
                        cmd = c;
                        break;
                    }
                    // the slot's CTA 0 answers within kIdleCap idle budgets; allow it two more
                    if (clock64() - t0 > (kIdleCap + 2) * a.idle_budget) break;
                    __nanosleep(500);
                }
            }
            s_cmd = cmd;
            if (cmd != kExit) {
                sp = sl->job;
                s_prec = sl->prec;
            }
        }
        __syncthreads();
        const unsigned cmd = s_cmd;
        if (cmd == kExit) return;
        last = cmd;
        if (s_prec == 0) {
            if (sp.nv == 2) run_chain<double, 1, 2, kThreads, false>(sp, s_cta, work, nullptr);
            else run_chain<double, 1, kVec, kThreads, false>(sp, s_cta, work, nullptr);
        } else {
            if (sp.nv == 2) run_chain<float, 1, 2, kThreads, false>(sp, s_cta, work, nullptr);
            else run_chain<float, 1, kVec, kThreads, false>(sp, s_cta, work, nullptr);
        }
        grid_barrier(sp, 9);  // every CTA of the slot is done with the job
        if (s_cta == 0 && threadIdx.x == 0) {
            __threadfence_system();
            st_release_sys_u32(a.done + s_slot, cmd);
        }
        __syncthreads();
    }
}

cudaError_t launch_server(const ServerArgs& a, int grid, int smem, cudaStream_t s)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_server_kernel);
    if (e != cudaSuccess) return e;
    ServerArgs q = a;
    void* args[] = {(void*)&q};
    return cudaLaunchCooperativeKernel((void*)gfmc_server_kernel, dim3(grid), dim3(kThreads), args, (size_t)smem, s);
}

cudaError_t server_max_ctas(int smem, int* out)
{
    cudaError_t e = allow_dynamic_smem((const void*)gfmc_server_kernel);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gfmc_server_kernel, kThreads, smem)) != cudaSuccess)
        return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *out = per_sm * sms;
    return cudaSuccess;
}

}  // namespace gfmc
