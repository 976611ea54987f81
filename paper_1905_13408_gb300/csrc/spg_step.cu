// Dispatch of the fused step over data dtypes, and the bounded-wait probe.
#include "spg_step_kernel.cuh"

namespace spg {

size_t step_smem_bytes_f32(const StepVariant &v);
size_t step_smem_bytes_bf16(const StepVariant &v);
cudaError_t step_configure_f32(const StepVariant &v, int *occ);
cudaError_t step_configure_bf16(const StepVariant &v, int *occ);
cudaError_t step_launch_f32(const StepVariant &v, int grid, const StepParams &p, cudaStream_t s);
cudaError_t step_launch_bf16(const StepVariant &v, int grid, const StepParams &p, cudaStream_t s);

namespace {

// Waits on a barrier that nothing ever arrives at, with the same bounded wait
// as the fused step: it must give up after `limit_ns` and record SPG_ETIMEOUT.
__global__ void timeout_probe_kernel(DevState *st, long long limit_ns)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0u, limit_ns);
    if (!ok && threadIdx.x == 0) atomicCAS(&st->err, 0, (int)SPG_ETIMEOUT);
}


}  // namespace

cudaError_t launch_timeout_probe(DevState *st, long long timeout_ns, cudaStream_t s)
{
    timeout_probe_kernel<<<1, 32, 0, s>>>(st, timeout_ns);
    return cudaGetLastError();
}

bool step_variant_supported(const StepVariant &v) { return step_smem_bytes_f32(v) != 0; }

size_t step_smem_bytes(const StepVariant &v) { return v.bf16 ? step_smem_bytes_bf16(v) : step_smem_bytes_f32(v); }

cudaError_t step_configure(const StepVariant &v, int *ctas_per_sm)
{
    return v.bf16 ? step_configure_bf16(v, ctas_per_sm) : step_configure_f32(v, ctas_per_sm);
}

cudaError_t step_launch(const StepVariant &v, int grid, const StepParams &p, cudaStream_t s)
{
    return v.bf16 ? step_launch_bf16(v, grid, p, s) : step_launch_f32(v, grid, p, s);
}

}  // namespace spg
