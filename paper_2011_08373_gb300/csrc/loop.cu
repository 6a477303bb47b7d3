// loop.cu — the loop kernel: Algorithm 1 (Section 2.4), one warp per
// program, over each program's conflict relation (see loop.cuh), and its
// host side.
#include <cuda_runtime.h>

#include <cstdint>

#include "loop.cuh"

namespace gr {

size_t loop_smem_bytes(bool simple) {
    return simple ? warp_smem<LoopWarpSimple>() * kSimpleWarps : warp_smem<LoopWarp>() * kLoopWarps;
}
uint32_t loop_threads(bool simple) { return simple ? kSimpleWarps * 32u : kLoopThreads; }

template <uint32_t WARPS, class LW>
__global__ void __launch_bounds__(WARPS * 32)
    k_loop(const uint8_t *__restrict__ arena, uint32_t n, gr_options opts, uint8_t *__restrict__ scratch,
           uint64_t scratch_bytes, gr_repair_result *__restrict__ out) {
    extern __shared__ uint4 loop_raw[];
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    LW &lw = *reinterpret_cast<LW *>(reinterpret_cast<uint8_t *>(loop_raw) + warp_smem<LW>() * warp);
    const ArenaView V = view(arena);
    uint32_t *ctrl = reinterpret_cast<uint32_t *>(scratch);
    const bool ok = launch_matches(V, n, scratch_bytes);
    // The first program's queue item, order entry and record come from the
    // queue counter (cleared before the relation kernel, which does not use
    // it) and the arena, so they are fetched before the wait below.
    uint32_t item = n;
    if (ok) {
        if (lane == 0) item = atomicAdd(&ctrl[3], 1u);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
        if (item < n) loop_load_record(lw, V, V.order[item]);
    }
    // Launched as a programmatic dependent of the relation kernel: its CTAs
    // may start while that kernel's last CTAs run, and wait here until it
    // has completed and its relation rows are visible (no wait when the
    // previous work in the stream was not a kernel that allows it).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if (!ok) {
        if (threadIdx.x == 0) atomicOr(&ctrl[1], kErrArgs);
        return;
    }
    const gr_witnesses *rel = reinterpret_cast<const gr_witnesses *>(scratch + V.h->scratch_rel_off);
    const uint32_t max_iters = opts.max_iters == 0 ? GR_MAX_ITERS : min(opts.max_iters, (uint32_t)GR_MAX_ITERS);
    const uint64_t deadline_ns = opts.deadline_us * 1000ull;
    for (bool first = true; item < n; first = false) {
        loop_program(lw, V, V.order[item], rel, opts, max_iters, deadline_ns, out, ctrl, first);
        if (lane == 0) item = atomicAdd(&ctrl[3], 1u);
        item = __shfl_sync(0xFFFFFFFFu, item, 0);
    }
}

cudaError_t configure_loop(uint32_t max_dynamic_smem) {
    (void)max_dynamic_smem;
    cudaError_t e = cudaFuncSetAttribute((const void *)k_loop<kLoopWarps, LoopWarp>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)loop_smem_bytes(false));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void *)k_loop<kSimpleWarps, LoopWarpSimple>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)loop_smem_bytes(true));
}

// The loop kernel may launch before the kernel ahead of it in the stream
// has finished (programmatic stream serialization): it waits for that
// kernel's completion itself, at its first instruction, so its launch and
// CTA placement overlap the relation kernel's tail.
cudaError_t launch_loop(const void *d_arena, uint32_t n, const gr_options &opts, void *d_scratch,
                        uint64_t scratch_bytes, gr_repair_result *d_out, uint32_t grid, bool simple, cudaStream_t st) {
    const uint8_t *a = static_cast<const uint8_t *>(d_arena);
    uint8_t *sc = static_cast<uint8_t *>(d_scratch);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (simple) {
        cfg.blockDim = dim3(kSimpleWarps * 32);
        cfg.dynamicSmemBytes = loop_smem_bytes(true);
        return cudaLaunchKernelEx(&cfg, k_loop<kSimpleWarps, LoopWarpSimple>, a, n, opts, sc, scratch_bytes, d_out);
    }
    cfg.blockDim = dim3(kLoopWarps * 32);
    cfg.dynamicSmemBytes = loop_smem_bytes(false);
    return cudaLaunchKernelEx(&cfg, k_loop<kLoopWarps, LoopWarp>, a, n, opts, sc, scratch_bytes, d_out);
}

}  // namespace gr
