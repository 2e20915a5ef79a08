// noalloc.cu -- a residual evaluation that allocates nothing.
//
// hofv_residual keeps its intermediate arrays (the extrapolated face values
// of the stabilisation, the per-face fluxes and, with HOFV_PREC_DF64, the
// state split into double-float pairs) in scratch memory that
// hofv_build_stencils allocated.  Some callers cannot let a library allocate
// device memory on their behalf: code that runs while a CUDA stream is being
// captured into a graph (where cudaMalloc is not permitted), real-time loops
// that forbid allocation after start-up, or host frameworks that own every
// device allocation through their own pool.  hofv_residual_noalloc serves
// them: those arrays live in a fixed file-scope device array, so the call
// itself calls no cudaMalloc, cudaFree or allocating library routine.
//
// Limits and caveats:
//   - The array holds kNoAllocScratchDoubles doubles (32 MiB), resident on
//     every GPU that loads this library until the process exits.  A mesh
//     needs n_cells * F * dim doubles for the extrapolated values (F = face
//     slots per cell: dim + 1 for triangles / tetrahedra, 2 dim for quads /
//     hexes, 8 for polygons), rounded up to a multiple of 32, plus
//     (internal + displacement + symmetry faces) * dim for the fluxes,
//     rounded up to 32, plus, with HOFV_PREC_DF64, (n_cells + mirror nodes)
//     * 4 (2-D) or 6 (3-D) for the split state, rounded up to 32.  Larger
//     meshes are rejected with HOFV_EINVAL.
//   - All calls share the one array: calls whose work overlaps on the GPU
//     (other streams, other threads, other contexts on the same device) race
//     on it and must be serialised by the caller.  Like every evaluation
//     call, it also writes buffers of its own hofv context (the extended
//     state of meshes with symmetry faces, the mirrored face values, the
//     inertia term), so it must also be ordered with the other evaluation
//     calls of the same context (hofv_residual, hofv_jvp, solves) issued
//     from other streams.
//   - The array keeps the previous call's contents.  Nothing in it has to
//     start at zero: every element the kernels read is written earlier in
//     the same call.
//   - The device address of the array is resolved with cudaGetSymbolAddress
//     on the first call on each device (with that device current) and again
//     whenever the device's current CUDA context has changed since (for
//     example after cudaDeviceReset); that first call should come before any
//     stream capture.
#include <cuda.h>

#include <mutex>

#include "hofv_internal.cuh"

namespace hofv {

constexpr int64_t kNoAllocScratchDoubles = (int64_t{32} << 20) / 8;

static __device__ __align__(256) double g_residual_scratch[kNoAllocScratchDoubles];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static double* g_scratch_addr[kMaxDevices] = {nullptr};
static CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};

typedef CUresult (*ctx_get_current_fn)(CUcontext*);

// the CUDA context current on the calling thread (nullptr if unknown)
static CUcontext current_context() {
  static ctx_get_current_fn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<ctx_get_current_fn>(p);
  }
  CUcontext ctx = nullptr;
  if (fn && fn(&ctx) != CUDA_SUCCESS) ctx = nullptr;
  return ctx;
}

// device address of g_residual_scratch on `device` in its current context
static int scratch_address(hofv_ctx* c, int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return fail(c, HOFV_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  int cur = -1;
  HOFV_CUDA(c, cudaGetDevice(&cur));
  if (cur != device) HOFV_CUDA(c, cudaSetDevice(device));
  const CUcontext ctx = current_context();
  cudaError_t e = cudaSuccess;
  if (!g_scratch_addr[device] || ctx != g_scratch_ctx[device]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_residual_scratch);
    if (e == cudaSuccess) {
      g_scratch_addr[device] = static_cast<double*>(p);
      g_scratch_ctx[device] = ctx;
    }
  }
  if (cur != device) cudaSetDevice(cur);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(residual scratch)");
  *out = g_scratch_addr[device];
  return 0;
}

static int64_t round32(int64_t n) { return ((n + 31) / 32) * 32; }

}  // namespace hofv

using namespace hofv;

extern "C" int hofv_residual_noalloc(hofv_ctx* c, const double* u, double* R) {
  if (!c) return HOFV_EINVAL;
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  if (!c->have_mat) return fail(c, HOFV_ESTATE, "hofv_set_material must come first");
  if (!u || !R) return fail(c, HOFV_EINVAL, "null vector");
  const int64_t n_ustar = round32(c->nc * c->nlf * c->dim);
  const int64_t n_flux = round32(std::max<int64_t>(c->nfid, 1) * c->dim);
  // split state: float4 slots, two doubles each
  const int64_t n_split =
      c->prec == HOFV_PREC_DF64 ? round32((c->nc + c->ng) * split4(c->dim) * 2) : 0;
  const int64_t need = n_ustar + n_flux + n_split;
  if (need > kNoAllocScratchDoubles)
    return fail(c, HOFV_EINVAL,
                "mesh too large for hofv_residual_noalloc: needs " + std::to_string(need) +
                    " doubles of scratch, the fixed array holds " +
                    std::to_string(kNoAllocScratchDoubles) + "; use hofv_residual");
  double* scratch = nullptr;
  const int rc = scratch_address(c, c->device, &scratch);
  if (rc != 0) return rc;
  c->mat.alpha = c->alpha;
  if (u == c->jv_u) {  // the caller may have changed u: the Jv linearisation is stale
    c->jv_cur++;
    c->jv_u = c->jv_R = nullptr;
  }
  DevMesh m = dev_mesh(c);
  if (n_split > 0) m.su = reinterpret_cast<float4*>(scratch + n_ustar + n_flux);
  launch_residual(m, c->mat, u, nullptr, nullptr, nullptr, R, scratch, scratch + n_ustar,
                  c->d_ubq, c->d_ubf, c->d_src, c->stream);
  HOFV_CUDA(c, cudaGetLastError());
  return HOFV_OK;
}
