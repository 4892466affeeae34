// Allocation-free entry point: density matrices from caller-supplied orbitals.
//
// Some callers cannot allocate GPU memory at the time they need this result: host codes
// whose memory is owned by a pre-sized pool of another framework, or real-time loops
// that forbid allocation after start-up (cudaMalloc may synchronise the device). This variant of the P/W contraction therefore
// uses a fixed scratch array that lives in the library image itself instead of a
// handle workspace.
//
// The scratch is a file-scope __device__ array of kNoAllocScratchDoubles doubles
// (16 MiB). Every GPU on which the library is loaded holds it until the process exits.
// All calls share it and each call overwrites the part it uses before reading it, so
// nothing has to start at zero; calls whose GPU work overlaps in time (different
// streams, or different host threads on the same device) race on it.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kNoAllocScratchDoubles = (size_t)1 << 21;  // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

std::mutex g_mu;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device. In host code the array's
// name is only a host-side stand-in, so the address has to be looked up once per device
// (with that device current).
int scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ELSI_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return ELSI_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return ELSI_OK;
}

}  // namespace

extern "C" int elsi_density_noalloc(int n_basis, int n_state, const double *evec,
                                    const double *occ, const double *eval, double *den_mat,
                                    double *edm, void *stream)
{
    if (n_basis < 1 || n_state < 1 || n_state > n_basis || !evec || !occ || !den_mat)
        return ELSI_ERR_ARG;
    if (edm && !eval) return ELSI_ERR_ARG;
    if ((size_t)n_basis * (size_t)n_state > kNoAllocScratchDoubles) return ELSI_ERR_TOO_LARGE;
    void *scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaError_t e = egb::density_pw<double>((cudaStream_t)stream, n_basis, n_state, evec, n_basis,
                                           occ, eval, den_mat, edm, static_cast<double *>(scratch));
    if (e != cudaSuccess) {
        // the cached address may belong to a context that no longer exists (a reset of
        // the device): look it up again on the next call
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < kMaxDevices) {
            std::lock_guard<std::mutex> lock(g_mu);
            g_scratch_ptr[dev] = nullptr;
        }
        return ELSI_ERR_CUDA;
    }
    return ELSI_OK;
}
