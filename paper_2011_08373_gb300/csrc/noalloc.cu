// noalloc.cu — gr_repair_packed_noalloc: the batched repair of a packed
// arena with its scratch in a fixed device array instead of a caller buffer.
//
// Some callers cannot allocate device memory at the point where they run the
// repair: code inside a host callback or a signal-safe path, a plug-in whose
// host forbids allocation after start-up, or a real-time loop that must not
// hit cudaMalloc's implicit device synchronisation and page-table work.  This
// entry point lets them repair a batch with only their own input (the packed
// arena) and output (the results) buffers.
//
// The scratch (address traces, per-segment masks and ranges, the conflict
// relations, the work-queue counters and the device error word) lives in
// `g_noalloc_scratch`, a file-scope static __device__ array of
// kNoAllocScratchBytes.  Every GPU that loads the library holds it until the
// process exits.  In host code that name is only a host-side stand-in for
// the symbol, not a device address, so the first call on each device (with
// that device current) looks the array's device address up with
// cudaGetSymbolAddress, checks the result and keeps it for that device; the
// kernels are given that address.  That first call should therefore come
// before any stream capture.  A cudaDeviceReset of the device discards the
// array with the context: do not call this entry point on that device again
// in the same process afterwards.  Every call reads the arena header back
// with a synchronising copy on its stream.  Every call shares the one array
// and it keeps the last call's contents: the control words are cleared on
// each call, everything else is rewritten before it is read.  Calls that
// overlap on the GPU (two streams, two host threads) race on the array and
// must not be issued; the host-side lock below only orders the enqueueing.
// The device error word stays inside the array and is not read back (the
// call does not wait for its kernels): device-side errors are not reported
// on this path; the library sizes every launch from the arena header, which
// this call checks first.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "engine.cuh"

namespace gr {

constexpr size_t kNoAllocScratchBytes = 64ull << 20;  // 64 MiB

static __device__ __align__(256) uint8_t g_noalloc_scratch[kNoAllocScratchBytes];

namespace {

std::mutex g_noalloc_mu;

// Per device, set up by its first call: the array's device address and the
// SM count (guarded by g_noalloc_mu).
constexpr int kNoAllocDevices = 64;
void *g_noalloc_ptr[kNoAllocDevices] = {};
int g_noalloc_sms[kNoAllocDevices] = {};

}  // namespace
void set_last_error(const char *msg);
namespace {

gr_status noalloc_fail(gr_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    set_last_error(buf);  // reported by gr_last_error()
    return code;
}

// Device address of the scratch array and the SM count of the current
// device: looked up by the first call on that device (which is current
// here), then kept.  Called with g_noalloc_mu held.
gr_status noalloc_setup(int *sms_out, void **ptr_out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(GR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kNoAllocDevices) return noalloc_fail(GR_ECUDA, "device index %d unsupported", dev);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(GR_ECUDA, "cudaGetSymbolAddress(g_noalloc_scratch): %s", cudaGetErrorString(e));
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return noalloc_fail(GR_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
        g_noalloc_sms[dev] = sms;
        g_noalloc_ptr[dev] = p;
    }
    *sms_out = g_noalloc_sms[dev];
    *ptr_out = g_noalloc_ptr[dev];
    return GR_OK;
}

}  // namespace

}  // namespace gr

using namespace gr;

extern "C" gr_status gr_repair_packed_noalloc(const void *d_arena, uint32_t n, const gr_options *opts,
                                              gr_repair_result *d_out, void *stream) {
    if (!d_arena || !d_out || n == 0) return noalloc_fail(GR_EINVAL, "NULL buffer or n == 0");
    if (reinterpret_cast<uintptr_t>(d_arena) % 256) return noalloc_fail(GR_EINVAL, "d_arena must be 256-byte aligned");
    gr_status s = validate_opts(opts);  // the same options gr_repair_packed accepts
    if (s != GR_OK) return s;
    std::lock_guard<std::mutex> g(g_noalloc_mu);
    int sms = 0;
    void *scratch = nullptr;
    if ((s = noalloc_setup(&sms, &scratch)) != GR_OK) return s;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the arena header says how much scratch the batch needs
    ArenaHeader h;
    cudaError_t e = cudaMemcpyAsync(&h, d_arena, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return noalloc_fail(GR_ECUDA, "reading the arena header: %s", cudaGetErrorString(e));
    if (h.magic != kArenaMagic || h.n_progs != n)
        return noalloc_fail(GR_EINVAL, "d_arena is not a packed arena of %u programs", n);
    if (h.scratch_bytes > kNoAllocScratchBytes)
        return noalloc_fail(GR_ECAPACITY, "batch needs %llu scratch bytes; the fixed array holds %llu",
                            (unsigned long long)h.scratch_bytes, (unsigned long long)kNoAllocScratchBytes);
    // the same launch as gr_repair_packed: the shapes gr_tune_packed recorded
    // for this arena, else the defaults
    const uint32_t skip = skip_bits(h);
    const LaunchCfg cfg = packed_launch_cfg(d_arena, n, skip, (h.flags & kArenaSimple) != 0, h.scratch_rel_off, &s);
    if (s != GR_OK) return noalloc_fail(s, "launch configuration failed");
    // the queue counters and the error word start at zero (cleared first)
    e = enqueue_repair(d_arena, n, opts_or_default(opts), scratch, kNoAllocScratchBytes, d_out, cfg,
                       (uint32_t)sms * 8u, true, true, st);
    if (e != cudaSuccess) return noalloc_fail(GR_ECUDA, "launch: %s", cudaGetErrorString(e));
    return GR_OK;
}
