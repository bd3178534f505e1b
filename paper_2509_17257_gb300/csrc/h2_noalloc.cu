// h2_matmul_noalloc: the product Y += alpha·A·X for callers that must not
// allocate device memory at call time.  Its scratch (gathered X, x̂, ŷ) lives
// in a fixed array compiled into this library instead of coming from
// cudaMalloc.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "h2_internal.cuh"

namespace {

// The scratch.  Every GPU that loads libh2.so reserves these bytes for the
// life of the process.
constexpr size_t kNoAllocScratchBytes = (size_t)H2_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // context the cached address belongs to

// Unique id of the calling thread's current context (0 if it cannot be
// read).  cudaDeviceReset destroys a device's primary context and the next
// runtime call creates a new one with a new id, in which the array has a new
// address; comparing ids keeps the cache from handing out the old one.  The
// driver functions come through the runtime's entry-point query, so the
// library does not link libcuda directly.
unsigned long long current_context_id() {
    using GetCurrent = int (*)(void**);
    using GetId = int (*)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        cudaDriverEntryPointQueryResult q1, q2;
        void* f1 = nullptr;
        void* f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            get_current = (GetCurrent)f1;
            get_id = (GetId)f2;
        }
        cudaGetLastError();
        looked_up = true;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the device address is
// looked up (with that device current) on the first call in a context and
// cached for that device until its context changes.
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        h2::set_error(std::string("h2_matmul_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return H2_E_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        h2::set_error("h2_matmul_noalloc: device index beyond 63");
        return H2_E_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    // ctx is 0 while no context is current on this thread yet, and always 0
    // where the driver's ids cannot be read (then the cache is per device)
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the device's context current if needed
        if (e != cudaSuccess || !p) {
            h2::set_error(std::string("h2_matmul_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return H2_E_CUDA;
        }
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = g_scratch_addr[dev];
    return 0;
}

}  // namespace

extern "C" int h2_matmul_noalloc(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                 int64_t m, int32_t dtype, void* stream) {
    if (!A || (m > 0 && (!X || !Y))) { h2::set_error("h2_matmul_noalloc: null argument"); return H2_E_BADARG; }
    if (m < 0 || ldx < m || ldy < m || m > ((int64_t)1 << 20)) {
        h2::set_error("h2_matmul_noalloc: bad m / leading dimension (0 <= m <= 2^20, ld >= m)");
        return H2_E_BADARG;
    }
    if (dtype != H2_F64 && dtype != H2_F32) {
        h2::set_error("h2_matmul_noalloc: dtype must be H2_F64 or H2_F32");
        return H2_E_UNSUPPORTED;
    }
    if (int rc = h2::refuse_complex(A, "h2_matmul_noalloc")) return rc;
    if (m == 0) return 0;
    if ((dtype == H2_F64 && !A->f64.built) || (dtype == H2_F32 && !A->f32.built)) {
        h2::set_error("h2_matmul_noalloc: this precision was not built for the matrix");
        return H2_E_UNSUPPORTED;
    }
    if (A->timing.on) {
        h2::set_error("h2_matmul_noalloc: disable h2_timing_enable first (it records events)");
        return H2_E_UNSUPPORTED;
    }
    if (!h2::is_device_pointer(X) || !h2::is_device_pointer(Y)) {
        h2::set_error("h2_matmul_noalloc: X and Y must be device memory");
        return H2_E_BADARG;
    }
    const size_t need = h2::product_scratch_bytes(A, m, dtype);
    if (need > kNoAllocScratchBytes) {
        h2::set_error("h2_matmul_noalloc: this product needs " + std::to_string(need) +
                      " bytes of scratch, more than the fixed " + std::to_string(kNoAllocScratchBytes) +
                      " bytes; use h2_matmul or fewer columns per call");
        return H2_E_UNSUPPORTED;
    }
    void* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    // The product clears the counters and flags at the end of the scratch
    // itself; every other scratch byte it reads (gathered X, x̂ and ŷ of all
    // clusters) is written earlier in the same product.
    return h2::matmul_in_scratch(A, alpha, X, ldx, Y, ldy, m, dtype, (cudaStream_t)stream, scratch);
}
