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

// Device address of g_noalloc_scratch on the current device.  In host code
// the array's name is only a host-side stand-in, so the device address is
// looked up once per device (with that device current) and cached.
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
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            h2::set_error(std::string("h2_matmul_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return H2_E_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return 0;
}

}  // namespace

extern "C" int h2_matmul_noalloc(h2_matrix* A, double alpha, const double* X, int64_t ldx, double* Y, int64_t ldy,
                                 int64_t m, int32_t dtype, void* stream) {
    if (!A || (m > 0 && (!X || !Y))) { h2::set_error("h2_matmul_noalloc: null argument"); return H2_E_BADARG; }
    if (m < 0 || ldx < m || ldy < m) { h2::set_error("h2_matmul_noalloc: bad m / leading dimension"); return H2_E_BADARG; }
    if (dtype != H2_F64 && dtype != H2_F32) {
        h2::set_error("h2_matmul_noalloc: dtype must be H2_F64 or H2_F32");
        return H2_E_UNSUPPORTED;
    }
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
