// Time-randomised control without any device allocation.
//
// bf_control_randomize() takes its sort scratch (64-bit keys and 32-bit
// indices for every sample) from the context's allocator, and it needs a
// context, whose creation allocates too.  Some callers cannot allocate device
// memory at the point where they need the control: code that runs inside a
// framework whose allocator owns all device memory, pipelines that fix their
// device-memory plan up front and must not grow it (or stall on an implicit
// synchronisation that cudaMalloc can cause), and callers working to a hard
// memory cap.  bf_control_randomize_static() serves them: it runs the same
// permutation kernels with the scratch held in the fixed array below, so it
// calls no cudaMalloc, cudaFree or other allocating routine.
//
// The array lives in the library's device code.  CUDA loads that code lazily
// by default, so the array (BF_STATIC_CONTROL_MAX samples of scratch, 12
// bytes per padded sample: 6 MiB) and the permutation kernels are placed in
// device memory by a set-up step: the first call on a device, or bf_init on
// that device, loads them and looks up the array's device address.  That
// first call may allocate through the driver; every later call allocates
// nothing.  The array then stays until the process exits, on every GPU that
// loaded it.  Every call shares it and finds the previous call's contents;
// the key kernel rewrites every entry it later reads, so nothing has to start
// at zero.  Two calls whose work overlaps on the GPU (for example on two
// streams) race on the array.
#include <mutex>

#include "bf_internal.h"
#include "runtime.h"

namespace bfi {

// padded sort length = next power of two >= n; keys (8 B) then indices (4 B)
constexpr uint64_t STATIC_CONTROL_PAD = 1ull << 19;
static_assert(BF_STATIC_CONTROL_MAX <= STATIC_CONTROL_PAD, "scratch sized for the maximum");
constexpr size_t STATIC_SCRATCH_BYTES = STATIC_CONTROL_PAD * (sizeof(uint64_t) + sizeof(uint32_t));

static __device__ __align__(256) unsigned char g_control_scratch[STATIC_SCRATCH_BYTES];

// Device address of the array per device.  In host code the name
// g_control_scratch is only a host-side stand-in, so kernels must be given
// this address, never the name.
static void* g_scratch_addr[64];
static std::mutex g_scratch_mu;

}  // namespace bfi

// With `device` current: looks the array's device address up (loading the
// module that holds it, on the first call) and, the first time that address
// is seen on the device, loads the permutation kernels too, so that no later
// call loads code.  The lookup runs on every call -- once the module is
// loaded it is a host-side table lookup -- so that after a cudaDeviceReset,
// which unloads the module, the address is taken afresh rather than reused.
bf_status bfi::static_control_setup(int device, void** addr)
{
    if (device < 0 || device >= 64) {
        set_error("device ordinal %d out of range", device);
        return BF_EINVAL;
    }
    std::lock_guard<std::mutex> g(g_scratch_mu);
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_control_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the control scratch");
    if (p != g_scratch_addr[device]) {
        e = preload_permute();
        if (e != cudaSuccess) return cuda_fail(e, "loading the permutation kernels");
        g_scratch_addr[device] = p;
    }
    if (addr) *addr = p;
    return BF_OK;
}

namespace bfi {

static bool on_device(const void* p, int device)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}

}  // namespace bfi

using namespace bfi;

extern "C" bf_status bf_control_randomize_static(const float* in, size_t n, uint64_t seed,
                                                 float* out, void* stream)
{
    if (!in || !out) { set_error("NULL argument"); return BF_EINVAL; }
    if (n == 0) return BF_OK;
    if (n > BF_STATIC_CONTROL_MAX) {
        set_error("bf_control_randomize_static: %zu samples exceed the fixed scratch of %d samples",
                  n, BF_STATIC_CONTROL_MAX);
        return BF_EINVAL;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (!on_device(in, dev) || !on_device(out, dev)) {
        set_error("bf_control_randomize_static: in and out must be memory of the current device %d", dev);
        return BF_EINVAL;
    }
    const char* a = reinterpret_cast<const char*>(in);
    const char* b = reinterpret_cast<const char*>(out);
    if (a < b + n * 4 && b < a + n * 4) { set_error("in and out overlap"); return BF_EINVAL; }
    void* scratch = nullptr;
    bf_status st = static_control_setup(dev, &scratch);
    if (st) return st;
    e = launch_permute(in, n, seed, out, scratch, static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "control randomisation (static scratch)");
}
