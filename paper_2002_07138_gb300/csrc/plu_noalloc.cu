// plu_lu_reorth_static: the re-orthogonalising panel LU (the same kernels as
// plu_lu_reorth) for callers that cannot allocate device memory.
//
// Who needs it: every other entry point works through a plu_ctx, and creating
// a context (and growing its workspace) calls cudaMalloc.  Some callers cannot
// do that: a host framework that has handed all of the GPU's memory to its own
// pool allocator (a raw cudaMalloc then fails or fragments the pool), plug-ins
// and embedded runtimes whose rules forbid allocating, and latency-critical
// loops that cannot pay for cudaMalloc / cudaFree, which may synchronise the
// whole device.  This entry point allocates nothing: its scratch memory (grid
// barrier word, per-CTA pivot candidates, U rows, row positions and the status
// word) lives in one file-scope device array of fixed size, kStaticBytes
// (2 MiB), which every GPU that loads the library holds until the process
// exits.  Hence the size limits: rows <= 65536 and cols <= 256.
//
// Set-up: the first call in each CUDA context of a device (the device
// current) looks up the device address of the array (cudaGetSymbolAddress)
// and the SM count; make that first call before any stream capture.  The
// cached address is tied to the context's unique id, so after a device reset
// (a new primary context, in which the module and its array may sit
// elsewhere) the next call repeats the set-up.  Every call shares the array and
// finds the previous call's contents there; the call clears what must start
// at zero (the status word and the barrier header).  Calls whose work overlaps
// on the GPU (on different streams, or from several host threads without
// ordering) race on the array and must not be issued.
#include "plu_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdarg>
#include <cstdio>
#include <mutex>

namespace {

constexpr size_t kStaticBytes = size_t(2) << 20;     // 2 MiB
constexpr int64_t kStaticMaxRows = 65536;
constexpr int kStaticMaxCols = 256;
constexpr size_t kStatusBytes = 256;                  // status word, then the panel scratch
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_plu_static_scratch[kStaticBytes];

struct DeviceSlot {
    bool ready = false;
    unsigned long long ctx_id = 0;   // unique id of the context the address belongs to
    char* base = nullptr;            // device address of g_plu_static_scratch on that device
    int num_sms = 0;
};
DeviceSlot g_slots[kMaxDevices];
std::mutex g_mutex;

// Unique id of the calling thread's current context (0 when the driver does
// not report one: the set-up then runs on every call).
unsigned long long current_ctx_id() {
    static PFN_cuCtxGetCurrent_v4000 get_cur = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 4000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(p);
        looked = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_cur || !get_id || get_cur(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
        return 0;
    return id;
}

plu_status say(char* err, size_t err_len, plu_status st, const char* fmt, ...) {
    if (err && err_len > 0) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(err, err_len, fmt, ap);
        va_end(ap);
    }
    return st;
}

}  // namespace

extern "C" plu_status plu_lu_reorth_static(void* cuda_stream, int64_t rows, int cols, double* X,
                                           int64_t ldx, char* err, size_t err_len) {
    if (err && err_len > 0) err[0] = '\0';
    if (!X || cols < 1 || rows < cols || ldx < rows)
        return say(err, err_len, PLU_EINVAL,
                   "plu_lu_reorth_static needs X != NULL, rows >= cols >= 1, ldx >= rows");
    if (rows > kStaticMaxRows || cols > kStaticMaxCols)
        return say(err, err_len, PLU_EINVAL,
                   "plu_lu_reorth_static takes at most %lld rows and %d columns (got %lld x %d): "
                   "its scratch is a fixed %zu-byte device array",
                   (long long)kStaticMaxRows, kStaticMaxCols, (long long)rows, cols, kStaticBytes);
    const size_t need = kStatusBytes + plu::panel_scratch_bytes(rows, cols);
    if (need > kStaticBytes)
        return say(err, err_len, PLU_EINVAL, "panel needs %zu bytes of scratch, the array has %zu",
                   need, kStaticBytes);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return say(err, err_len, PLU_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return say(err, err_len, PLU_EINVAL, "device %d out of range", dev);
    DeviceSlot slot;
    {
        std::lock_guard<std::mutex> lock(g_mutex);
        // 0 before the runtime has made the device's primary context current
        const unsigned long long id = current_ctx_id();
        if (!g_slots[dev].ready || id == 0 || g_slots[dev].ctx_id != id) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_plu_static_scratch);
            if (e != cudaSuccess)
                return say(err, err_len, PLU_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            int sms = 0;
            e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess)
                return say(err, err_len, PLU_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
            g_slots[dev].base = static_cast<char*>(ptr);
            g_slots[dev].num_sms = sms;
            g_slots[dev].ctx_id = current_ctx_id();   // the lookup made the context current
            g_slots[dev].ready = true;
        }
        slot = g_slots[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    int* status = reinterpret_cast<int*>(slot.base);
    void* scratch = slot.base + kStatusBytes;
    e = cudaMemsetAsync(status, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = plu::launch_panel_lu(rows, cols, X, ldx, 0, nullptr, nullptr, 0, 0, nullptr, 0, 0,
                                 nullptr, scratch, status, 16LL << 20, slot.num_sms, s);
    if (e != cudaSuccess) return say(err, err_len, PLU_ECUDA, "launch: %s", cudaGetErrorString(e));
    int h_status = 0;
    e = cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return say(err, err_len, PLU_ECUDA, "sync: %s", cudaGetErrorString(e));
    if (h_status == plu::DEV_TIMEOUT)
        return say(err, err_len, PLU_ETIMEOUT, "a device-side wait ran out of its budget");
    if (h_status != plu::DEV_OK)
        return say(err, err_len, PLU_ENUMERIC, "non-finite value in the panel");
    return PLU_OK;
}
