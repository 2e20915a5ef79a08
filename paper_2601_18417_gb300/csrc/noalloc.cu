// noalloc.cu -- a residual evaluation that allocates nothing.
//
// hofv_residual keeps its two intermediate arrays (the extrapolated face
// values of the stabilisation and the per-face fluxes) in scratch memory that
// hofv_build_stencils allocated.  Some callers cannot let a library allocate
// device memory on their behalf: code that runs while a CUDA stream is being
// captured into a graph (where cudaMalloc is not permitted), real-time loops
// that forbid allocation after start-up, or host frameworks that own every
// device allocation through their own pool.  hofv_residual_noalloc serves
// them: its scratch is a fixed file-scope device array, so the call itself
// calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and caveats:
//   - The array holds kNoAllocScratchDoubles doubles (32 MiB), resident on
//     every GPU that loads this library until the process exits.  Meshes
//     whose scratch (n_cells * 2 dim * dim + n_faces_with_stencil * dim
//     doubles) does not fit are rejected with HOFV_EINVAL.
//   - All calls share the one array: calls whose work overlaps on the GPU
//     (other streams, other threads, other contexts on the same device) race
//     on it and must be serialised by the caller.
//   - The array keeps the previous call's contents.  Nothing in it has to
//     start at zero: every element the kernels read is written earlier in
//     the same call.
//   - The device address of the array is resolved with cudaGetSymbolAddress
//     on the first call on each device (with that device current), so that
//     first call should come before any stream capture.
#include <mutex>

#include "hofv_internal.cuh"

namespace hofv {

constexpr int64_t kNoAllocScratchDoubles = (int64_t{32} << 20) / 8;

static __device__ __align__(256) double g_residual_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static double* g_scratch_addr[kMaxDevices] = {nullptr};

// device address of g_residual_scratch on `device`, resolved once
static int scratch_address(hofv_ctx* c, int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return fail(c, HOFV_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[device]) {
    int cur = -1;
    HOFV_CUDA(c, cudaGetDevice(&cur));
    if (cur != device) HOFV_CUDA(c, cudaSetDevice(device));
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (cur != device) cudaSetDevice(cur);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(residual scratch)");
    g_scratch_addr[device] = static_cast<double*>(p);
  }
  *out = g_scratch_addr[device];
  return 0;
}

}  // namespace hofv

using namespace hofv;

extern "C" int hofv_residual_noalloc(hofv_ctx* c, const double* u, double* R) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (!c->have_mat) return fail(c, HOFV_ESTATE, "hofv_set_material must come first");
  if (!u || !R) return fail(c, HOFV_EINVAL, "null vector");
  const int64_t n_ustar = ((c->nc * c->nlf * c->dim + 31) / 32) * 32;
  const int64_t n_flux = std::max<int64_t>(c->nfid, 1) * c->dim;
  if (n_ustar + n_flux > kNoAllocScratchDoubles)
    return fail(c, HOFV_EINVAL,
                "mesh too large for hofv_residual_noalloc: needs " +
                    std::to_string(n_ustar + n_flux) + " doubles of scratch, the fixed array holds " +
                    std::to_string(kNoAllocScratchDoubles) + "; use hofv_residual");
  double* scratch = nullptr;
  const int rc = scratch_address(c, c->device, &scratch);
  if (rc != 0) return rc;
  c->mat.alpha = c->alpha;
  launch_residual(dev_mesh(c), c->mat, u, nullptr, nullptr, nullptr, R, scratch, scratch + n_ustar,
                  c->d_ubq, c->d_ubf, c->d_src, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}
