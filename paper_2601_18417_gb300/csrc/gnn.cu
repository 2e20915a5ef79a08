// gnn.cu -- learned graph-network preconditioner (no counterpart in the
// paper): inference inside flexible GMRES and training by the library's own
// forward / backward kernels.
//
// Network (nodes = cells, neighbours = face neighbours, symmetric weights
// w_ij = a_ij / sqrt(D_i D_j) from the compact approximate Jacobian):
//   x_i  = [v_i / s_v, z_i / s_z, f_disp_i, f_trac_i, 0..]   (16)
//   h0_i = relu(W0 x_i + b0)                                 (64)
//   m_i  = sum_j w_ij h_j ; h_i += relu(Wl [h_i; m_i] + bl)  (4 layers)
//   y_i  = Wd h_i + bd ; z_out = z + s_z y
// with z = P_AJ^{-1} v.  s_v, s_z are the RMS of v and z, so the map is
// equivariant to scaling of v.  Training minimises
//   sum_i |z_out_i - delta_i|^2 / sum_i |delta_i|^2
// over (residual, Newton correction) pairs recorded by the solver.
//
// Every node-wise GEMM (the encoder and its weight gradient, the message-
// passing layers forward and both backward products) runs on the 5th-
// generation tensor cores: tcgen05.mma with BF16 operands in shared memory
// and FP32 accumulators in tensor memory, 128 nodes a tile; the decoder
// (64 -> d) is FP32 FMAs.  The message passing is a gather over the
// symmetric graph, so its transpose in the backward pass is the same gather
// (no atomics); weight gradients are accumulated per block and reduced in
// block order (deterministic).
#include <cuda_bf16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <vector>

#include "hofv_internal.cuh"

namespace hofv {

namespace {

constexpr int GH = 64;          // hidden width
constexpr int GF = 16;          // input features (padded)
constexpr int GL = 4;           // message-passing layers
typedef __nv_bfloat16 bf16;

struct Gnn {
  int dim = 0, nlf = 0;
  int64_t n = 0, ntiles = 0, npad = 0;
  int64_t P = 0;                // parameter count
  int64_t off_W0, off_b0, off_W[GL], off_b[GL], off_Wd, off_bd;
  // graph
  float* w = nullptr;           // [n][nlf]
  float* bnd = nullptr;         // [n][2]
  // parameters
  float* theta = nullptr;       // FP32 master
  float* grad = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  bf16* W0b = nullptr;          // [64][16]
  bf16* Wb = nullptr;           // [GL][64][128]
  int64_t adam_t = 0;
  // activations
  bf16* x = nullptr;            // [npad][16]
  bf16* h = nullptr;            // [GL+1][npad][64]
  bf16* a = nullptr;            // [GL+1][npad][64] pre-activations
  float* dh0 = nullptr;         // [npad][64]
  float* dh1 = nullptr;
  float* dm = nullptr;          // [npad][64]
  float* part = nullptr;        // [gblocks][64*128 + 64]
  double* scal = nullptr;       // 0 |v|, 1 |z|, 2 s_v, 3 s_z, 4 |delta|^2, 5 loss
  int gblocks = 0;
  // recorded training pairs (residual, correction) and cached z_AJ
  std::vector<double*> pr, pd, pz;
  std::vector<void*> allocs;
};

template <typename T>
int galloc(hofv_ctx* c, Gnn* g, T** p, int64_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, sizeof(T) * count + 16);
  if (e != cudaSuccess) return fail(c, HOFV_ENOMEM, "learned preconditioner: out of device memory");
  g->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return 0;
}

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// ---------------------------------------------------------------------
// graph: symmetric weights and boundary fractions
// ---------------------------------------------------------------------
__global__ void k_gnn_graph(int nlf, int64_t n, int64_t nfi, const double* __restrict__ diag,
                            const int32_t* __restrict__ col, const double* __restrict__ off,
                            const int32_t* __restrict__ cface, const int64_t* __restrict__ cf,
                            float* w, float* bnd) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int nd = 0, nt = 0, nf = 0;  // the cell's faces: displacement (or symmetry), traction, all
  for (int k = 0; k < nlf; ++k) {
    const int32_t j = col[i * nlf + k];
    w[i * nlf + k] = j >= 0 ? (float)(off[i * nlf + k] / sqrt(diag[i] * diag[j])) : 0.f;
    if (cf[i * nlf + k] < 0) continue;  // a polygon / polyhedron slot without a face
    ++nf;
    const int32_t code = cface[i * nlf + k];
    if (code == 0) ++nt;
    else if (code > 0 && code - 1 >= nfi) ++nd;
  }
  bnd[2 * i] = (float)nd / nf;
  bnd[2 * i + 1] = (float)nt / nf;
}

// rms scales from the norms: s = |x| / sqrt(count), 1 when the vector is zero
__global__ void k_gnn_scales(double* scal, double inv_sqrt_count) {
  for (int k = 0; k < 2; ++k) {
    const double s = scal[k] * inv_sqrt_count;
    scal[2 + k] = s > 0.0 ? s : 1.0;
  }
}

__global__ void k_square(double* x) { x[0] = x[0] * x[0]; }


// ---------------------------------------------------------------------
// the same layer on the 5th-generation tensor cores: 128 nodes a block, the
// operands [h | m] (128 x 128) and W (64 x 128) in shared memory in the
// canonical K-major layout without swizzle (8-row x 16-byte core matrices;
// K-direction core stride kTcLboA / kTcLboB, row-group stride 128 bytes),
// one thread issuing eight tcgen05.mma of K = 16 into a 128 x 64 FP32
// accumulator in tensor memory (64 columns), completion signalled on an
// mbarrier, and each warp reading its 32 rows back with tcgen05.ld.
// ---------------------------------------------------------------------
constexpr int kTcRows = 128;                       // nodes per block (MMA M)
constexpr int kTcLboA = kTcRows * 16;              // bytes between K-adjacent core matrices of A
constexpr int kTcLboB = GH * 16;                   // ... of W
constexpr int kTcSmem = kTcRows * 2 * GH * 2 + GH * 2 * GH * 2;  // A then W, bytes
constexpr long long kTcSpin = 1LL << 26;           // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (row, k) of a K-major operand with lbo bytes
// between K-adjacent core matrices and 128 between row-adjacent ones
__device__ __forceinline__ int tc_off(int row, int k, int lbo) {
  return (k >> 3) * lbo + (row >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor: start, leading (K) and stride (row
// group) byte offsets in 16-byte units, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__global__ void __launch_bounds__(128)
    k_gnn_layer_tc(int nlf, int64_t n, int64_t npad, const bf16* __restrict__ hin,
                   const int32_t* __restrict__ col, const float* __restrict__ w,
                   const bf16* __restrict__ Wb, const float* __restrict__ b, bf16* aout,
                   bf16* hout) {
  extern __shared__ __align__(1024) uint8_t tsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  uint8_t* sA = tsm;
  uint8_t* sW = tsm + kTcRows * 2 * GH * 2;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t base = (int64_t)blockIdx.x * kTcRows;
  // [h | m] of the tile's nodes (zero past the last node)
  for (int e = tid; e < kTcRows * (GH / 8); e += 128) {
    const int r = e / (GH / 8), ch = e % (GH / 8);
    const int64_t i = base + r;
    float mv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint4 own = make_uint4(0, 0, 0, 0);
    if (i < n) {
      own = *reinterpret_cast<const uint4*>(hin + i * GH + ch * 8);
      for (int k = 0; k < nlf; ++k) {
        const int32_t j = col[i * nlf + k];
        if (j < 0) continue;
        const float wk = w[i * nlf + k];
        const uint4 hv = *reinterpret_cast<const uint4*>(hin + (int64_t)j * GH + ch * 8);
        const bf16* hb = reinterpret_cast<const bf16*>(&hv);
#pragma unroll
        for (int q = 0; q < 8; ++q) mv[q] = fmaf(wk, __bfloat162float(hb[q]), mv[q]);
      }
    }
    *reinterpret_cast<uint4*>(sA + tc_off(r, ch * 8, kTcLboA)) = own;
    __align__(16) bf16 mb[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) mb[q] = __float2bfloat16_rn(mv[q]);
    *reinterpret_cast<uint4*>(sA + tc_off(r, GH + ch * 8, kTcLboA)) =
        *reinterpret_cast<const uint4*>(mb);
  }
  for (int e = tid; e < GH * (2 * GH / 8); e += 128) {
    const int r = e / (2 * GH / 8), ch = e % (2 * GH / 8);
    *reinterpret_cast<uint4*>(sW + tc_off(r, ch * 8, kTcLboB)) =
        *reinterpret_cast<const uint4*>(Wb + r * 2 * GH + ch * 8);
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
        smem_addr(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // the generic-proxy stores above become visible to the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  if (tid == 0) {
    // kind::f16: D FP32, A and B BF16, both K-major, N = 64, M = 128
    const uint32_t idesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GH / 8) << 17) | ((uint32_t)(kTcRows / 16) << 24);
#pragma unroll
    for (int ks = 0; ks < 2 * GH / 16; ++ks) {
      const uint64_t ad = tc_desc(smem_addr(sA) + ks * 2 * kTcLboA, kTcLboA, 128);
      const uint64_t bd = tc_desc(smem_addr(sW) + ks * 2 * kTcLboB, kTcLboB, 128);
      asm volatile(
          "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
          "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
          "l"(ad), "l"(bd), "r"(idesc), "r"(ks > 0 ? 1u : 0u));
    }
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_addr(&mbar)));
  }
  uint32_t done = 0;
  for (long long it = 0; it < kTcSpin && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(&mbar)));
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int r = tid;  // warp w reads rows 32 w .. 32 w + 31 (its lane quadrant)
  const int64_t row = base + r;
  float acc[GH];
  if (done) {
    uint32_t v[GH];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,"
        "%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,"
        "%61,%62,%63}, [%64];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
          "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
          "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
          "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]),
          "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]),
          "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]),
          "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
          "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]),
          "=r"(v[62]), "=r"(v[63])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < GH; ++j) acc[j] = __uint_as_float(v[j]);
  } else {  // the product did not complete: NaN, which the solver rejects
#pragma unroll
    for (int j = 0; j < GH; ++j) acc[j] = __int_as_float(0x7fc00000);
  }
  if (row < npad) {
#pragma unroll
    for (int c8 = 0; c8 < GH / 8; ++c8) {
      const uint4 hv = *reinterpret_cast<const uint4*>(sA + tc_off(r, c8 * 8, kTcLboA));
      const bf16* hb = reinterpret_cast<const bf16*>(&hv);
      __align__(16) bf16 ab[8], ob[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float pre = acc[c8 * 8 + q] + b[c8 * 8 + q];
        ab[q] = __float2bfloat16_rn(pre);
        ob[q] = __float2bfloat16_rn(__bfloat162float(hb[q]) + relu(pre));
      }
      *reinterpret_cast<uint4*>(aout + row * GH + c8 * 8) = *reinterpret_cast<const uint4*>(ab);
      *reinterpret_cast<uint4*>(hout + row * GH + c8 * 8) = *reinterpret_cast<const uint4*>(ob);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------------
// backward of one layer on the tensor cores, 128 nodes a tile, persistent
// over tiles:
//   [dself | dm] (128 nodes x 128) = dpre (128 x 64) W (64 x 128)   (GEMM 1)
//   dW^T (128 x 64) += X^T (128 x 128 nodes) dpre (128 nodes x 64)   (GEMM 2)
// with dpre = dh_out where the pre-activation is positive.  Operands in the
// same canonical K-major layout as the forward: A of GEMM 1 = dpre (rows
// nodes, K = outputs), B = W^T (rows inputs, K = outputs); A of GEMM 2 = X^T
// (rows inputs, K = nodes), B = dpre^T (rows outputs, K = nodes).  Tensor
// memory: columns 0-127 GEMM 1 (per tile), 128-191 GEMM 2 (accumulated over
// the block's tiles, read once at the end as the block's dW partial).
// ---------------------------------------------------------------------
constexpr int kTcBwdSmem = 2 * GH * kTcRows * 2     // X^T
                           + kTcRows * GH * 2       // dpre
                           + GH * kTcRows * 2       // dpre^T
                           + 2 * GH * GH * 2;       // W^T

__device__ __forceinline__ void tc_ld64(uint32_t taddr, float* out) {
  uint32_t v[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,"
      "%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,"
      "%61,%62,%63}, [%64];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
        "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]),
        "=r"(v[38]), "=r"(v[39]), "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]),
        "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]), "=r"(v[48]), "=r"(v[49]),
        "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
        "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]),
        "=r"(v[62]), "=r"(v[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 64; ++j) out[j] = __uint_as_float(v[j]);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

// bounded wait for the commit of phase `parity`; 1 when it completed
__device__ __forceinline__ uint32_t tc_wait(const uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < kTcSpin && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_addr(mbar)), "r"(parity));
  }
  return done;
}

__global__ void __launch_bounds__(128)
    k_gnn_layer_bwd_tc(int nlf, int64_t n, int64_t ntc, const bf16* __restrict__ hin,
                       const bf16* __restrict__ a, const int32_t* __restrict__ col,
                       const float* __restrict__ w, const bf16* __restrict__ Wb,
                       const float* __restrict__ dh_out, float* dnext, float* dm, float* part,
                       int part_stride) {
  extern __shared__ __align__(1024) uint8_t bsm[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  uint8_t* sXT = bsm;
  uint8_t* sD = sXT + 2 * GH * kTcRows * 2;
  uint8_t* sDT = sD + kTcRows * GH * 2;
  uint8_t* sWT = sDT + GH * kTcRows * 2;
  constexpr int kLbo128 = kTcRows * 16, kLbo64 = GH * 16;
  const int tid = threadIdx.x, warp = tid >> 5;
  // W^T: row i (input feature), K = output o
  for (int e = tid; e < GH * 2 * GH; e += 128) {
    const int o = e / (2 * GH), i = e % (2 * GH);
    *reinterpret_cast<bf16*>(sWT + tc_off(i, o, kLbo128)) = Wb[e];
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
        smem_addr(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  const uint32_t id1 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(2 * GH / 8) << 17) |
                       ((uint32_t)(kTcRows / 16) << 24);  // M 128, N 128
  const uint32_t id2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GH / 8) << 17) |
                       ((uint32_t)(kTcRows / 16) << 24);  // M 128, N 64
  float gb = 0.f;  // db of output feature tid (< 64)
  uint32_t ok = 1, iter = 0;
  for (int64_t tile = blockIdx.x; tile < ntc && ok; tile += gridDim.x, ++iter) {
    const int64_t base = tile * kTcRows;
    // X^T: [h | m] of the tile's nodes, transposed (rows = input features)
    for (int e = tid; e < kTcRows * (GH / 8); e += 128) {
      const int r = e / (GH / 8), ch = e % (GH / 8);
      const int64_t i = base + r;
      float mv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      uint4 own = make_uint4(0, 0, 0, 0);
      if (i < n) {
        own = *reinterpret_cast<const uint4*>(hin + i * GH + ch * 8);
        for (int k = 0; k < nlf; ++k) {
          const int32_t j = col[i * nlf + k];
          if (j < 0) continue;
          const float wk = w[i * nlf + k];
          const uint4 hv = *reinterpret_cast<const uint4*>(hin + (int64_t)j * GH + ch * 8);
          const bf16* hb = reinterpret_cast<const bf16*>(&hv);
#pragma unroll
          for (int q = 0; q < 8; ++q) mv[q] = fmaf(wk, __bfloat162float(hb[q]), mv[q]);
        }
      }
      const bf16* ob = reinterpret_cast<const bf16*>(&own);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        *reinterpret_cast<bf16*>(sXT + tc_off(ch * 8 + q, r, kLbo128)) = ob[q];
        *reinterpret_cast<bf16*>(sXT + tc_off(GH + ch * 8 + q, r, kLbo128)) =
            __float2bfloat16_rn(mv[q]);
      }
    }
    // dpre and its transpose
    for (int e = tid; e < kTcRows * GH; e += 128) {
      const int r = e / GH, f = e % GH;
      const int64_t i = base + r;
      float d = 0.f;
      if (i < n && __bfloat162float(a[i * GH + f]) > 0.f) d = dh_out[i * GH + f];
      const bf16 db = __float2bfloat16_rn(d);
      *reinterpret_cast<bf16*>(sD + tc_off(r, f, kLbo128)) = db;
      *reinterpret_cast<bf16*>(sDT + tc_off(f, r, kLbo64)) = db;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < GH / 16; ++ks)
        tc_mma(tmem, tc_desc(smem_addr(sD) + ks * 2 * kLbo128, kLbo128, 128),
               tc_desc(smem_addr(sWT) + ks * 2 * kLbo128, kLbo128, 128), id1, ks > 0 ? 1u : 0u);
#pragma unroll
      for (int ks = 0; ks < kTcRows / 16; ++ks)
        tc_mma(tmem + 2 * GH, tc_desc(smem_addr(sXT) + ks * 2 * kLbo128, kLbo128, 128),
               tc_desc(smem_addr(sDT) + ks * 2 * kLbo64, kLbo64, 128), id2,
               (ks > 0 || iter > 0) ? 1u : 0u);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&mbar)));
    }
    if (tid < GH)
      for (int r = 0; r < kTcRows; ++r)
        gb += __bfloat162float(*reinterpret_cast<const bf16*>(sDT + tc_off(tid, r, kLbo64)));
    ok = tc_wait(&mbar, iter & 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int64_t i = base + tid;  // warp w holds rows 32 w .. 32 w + 31
    float acc[64];
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    if (ok) tc_ld64(lane_base, acc);
    if (i < n) {
      for (int c = 0; c < GH; ++c)
        dnext[i * GH + c] = ok ? dh_out[i * GH + c] + acc[c] : __int_as_float(0x7fc00000);
    }
    if (ok) tc_ld64(lane_base + GH, acc);
    if (i < n) {
      for (int c = 0; c < GH; ++c) dm[i * GH + c] = ok ? acc[c] : __int_as_float(0x7fc00000);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // operands and tensor-memory columns 0-127 are reused by the next tile
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  // the block's dW partial: thread tid = input feature i reads dW^T[i][0..63]
  float* pp = part + (int64_t)blockIdx.x * part_stride;
  {
    float acc[64];
    if (iter > 0 && ok) {
      tc_ld64(tmem + ((uint32_t)(warp * 32) << 16) + 2 * GH, acc);
    } else {
#pragma unroll
      for (int j = 0; j < 64; ++j) acc[j] = iter > 0 ? __int_as_float(0x7fc00000) : 0.f;
    }
    for (int o = 0; o < GH; ++o) pp[o * 2 * GH + tid] = acc[o];
  }
  if (tid < GH) pp[GH * 2 * GH + tid] = ok ? gb : __int_as_float(0x7fc00000);
  if (!ok) tc_wait(&mbar, (iter - 1) & 1);  // a late commit: wait again (bounded) before freeing
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem));
}

// ---------------------------------------------------------------------
// the encoder on the tensor cores: x (128 nodes x 16 features) times W0^T
// (16 x 64) as one tcgen05.mma of K = 16 into 64 tensor-memory columns
// ---------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(128)
    k_gnn_encode_tc(int64_t n, int64_t npad, int64_t ntc, const double* __restrict__ v,
                    const double* __restrict__ z, const float* __restrict__ bnd,
                    const double* __restrict__ scal, const bf16* __restrict__ W0b,
                    const float* __restrict__ b0, bf16* xg, bf16* a0, bf16* h0) {
  __shared__ __align__(1024) uint8_t sx[kTcRows * GF * 2];  // A: rows nodes, K features
  __shared__ __align__(1024) uint8_t sw[GH * GF * 2];       // B: rows outputs, K features
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  constexpr int kLboX = kTcRows * 16, kLboW = GH * 16;
  const int tid = threadIdx.x, warp = tid >> 5;
  const double isv = 1.0 / scal[2], isz = 1.0 / scal[3];
  for (int e = tid; e < GH * GF; e += 128)
    *reinterpret_cast<bf16*>(sw + tc_off(e / GF, e % GF, kLboW)) = W0b[e];
  if (warp == 0) {  // once per block: the grid is a few blocks an SM, persistent over tiles
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(
        smem_addr(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GH / 8) << 17) |
                         ((uint32_t)(kTcRows / 16) << 24);  // M 128, N 64
  uint32_t ok = 1, iter = 0;
  for (int64_t tile = blockIdx.x; tile < ntc && ok; tile += gridDim.x, ++iter) {
    const int64_t base = tile * kTcRows;
    // one node per thread: its 16 features
    {
      const int r = tid;
      const int64_t i = base + r;
      __align__(16) bf16 xb[GF];
#pragma unroll
      for (int f = 0; f < GF; ++f) {
        float val = 0.f;
        if (i < n) {
          if (f < DIM) val = (float)(v[f * n + i] * isv);
          else if (f < 2 * DIM) val = (float)(z[(f - DIM) * n + i] * isz);
          else if (f < 2 * DIM + 2) val = bnd[2 * i + (f - 2 * DIM)];
        }
        xb[f] = __float2bfloat16_rn(val);
      }
#pragma unroll
      for (int c8 = 0; c8 < GF / 8; ++c8) {
        const uint4 q = reinterpret_cast<const uint4*>(xb)[c8];
        *reinterpret_cast<uint4*>(sx + tc_off(r, c8 * 8, kLboX)) = q;
        if (i < npad) *reinterpret_cast<uint4*>(xg + i * GF + c8 * 8) = q;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      tc_mma(tmem, tc_desc(smem_addr(sx), kLboX, 128), tc_desc(smem_addr(sw), kLboW, 128), idesc,
             0u);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&mbar)));
    }
    ok = tc_wait(&mbar, iter & 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float acc[GH];
    if (ok) {
      tc_ld64(tmem + ((uint32_t)(warp * 32) << 16), acc);
    } else {  // the product did not complete: NaN, which the solver rejects
#pragma unroll
      for (int j = 0; j < GH; ++j) acc[j] = __int_as_float(0x7fc00000);
    }
    const int64_t row = base + tid;
    if (row < npad) {
#pragma unroll
      for (int c8 = 0; c8 < GH / 8; ++c8) {
        __align__(16) bf16 ab[8], hb[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float pre = acc[c8 * 8 + q] + b0[c8 * 8 + q];
          ab[q] = __float2bfloat16_rn(pre);
          hb[q] = __float2bfloat16_rn(relu(pre));
        }
        *reinterpret_cast<uint4*>(a0 + row * GH + c8 * 8) = *reinterpret_cast<const uint4*>(ab);
        *reinterpret_cast<uint4*>(h0 + row * GH + c8 * 8) = *reinterpret_cast<const uint4*>(hb);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the operand and the accumulator are reused by the next tile
  }
  if (!ok) tc_wait(&mbar, (iter - 1) & 1);  // a late commit: wait again (bounded) before freeing
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem));
}

// ---------------------------------------------------------------------
// encoder backward on the tensor cores (persistent over 128-node tiles):
// dW0 (64 x 16) += dpre0^T (64 x 128 nodes) x (128 nodes x 16), as an
// M = 128 product whose rows 64-127 are zero, N = 16, accumulated in 16
// tensor-memory columns across the block's tiles; db0 from the same dpre0
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    k_gnn_encode_bwd_tc(int64_t n, int64_t npad, int64_t ntc, const bf16* __restrict__ xg,
                        const bf16* __restrict__ a0, const float* __restrict__ dh, float* part,
                        int part_stride) {
  __shared__ __align__(1024) uint8_t sA[kTcRows * kTcRows * 2];  // dpre0^T, rows 64.. zero
  __shared__ __align__(1024) uint8_t sB[GF * kTcRows * 2];       // x^T: rows features
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  constexpr int kLboA = kTcRows * 16, kLboB = GF * 16;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int e = tid; e < kTcRows * kTcRows / 8; e += 128)
    reinterpret_cast<uint4*>(sA)[e] = make_uint4(0, 0, 0, 0);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(
        smem_addr(&tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tslot;
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GF / 8) << 17) |
                         ((uint32_t)(kTcRows / 16) << 24);  // M 128, N 16
  float gb = 0.f;
  uint32_t ok = 1, iter = 0;
  for (int64_t tile = blockIdx.x; tile < ntc && ok; tile += gridDim.x, ++iter) {
    const int64_t base = tile * kTcRows;
    for (int e = tid; e < kTcRows * GH; e += 128) {
      const int r = e / GH, f = e % GH;
      const int64_t i = base + r;
      float d = 0.f;
      if (i < n && __bfloat162float(a0[i * GH + f]) > 0.f) d = dh[i * GH + f];
      *reinterpret_cast<bf16*>(sA + tc_off(f, r, kLboA)) = __float2bfloat16_rn(d);
    }
    for (int e = tid; e < kTcRows * GF; e += 128) {
      const int r = e / GF, f = e % GF;
      const int64_t i = base + r;
      *reinterpret_cast<bf16*>(sB + tc_off(f, r, kLboB)) =
          i < npad ? xg[i * GF + f] : __float2bfloat16_rn(0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kTcRows / 16; ++ks)
        tc_mma(tmem, tc_desc(smem_addr(sA) + ks * 2 * kLboA, kLboA, 128),
               tc_desc(smem_addr(sB) + ks * 2 * kLboB, kLboB, 128), idesc,
               (ks > 0 || iter > 0) ? 1u : 0u);
      asm volatile(
          "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
              smem_addr(&mbar)));
    }
    if (tid < GH)
      for (int r = 0; r < kTcRows; ++r)
        gb += __bfloat162float(*reinterpret_cast<const bf16*>(sA + tc_off(tid, r, kLboA)));
    ok = tc_wait(&mbar, iter & 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the operands are rewritten by the next tile
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  float* pp = part + (int64_t)blockIdx.x * part_stride;
  if (warp < 2) {  // rows 0-63: dW0[o][0..15], o = tid
    uint32_t v[GF];
    if (iter > 0 && ok) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
          "%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    } else {
#pragma unroll
      for (int j = 0; j < GF; ++j) v[j] = iter > 0 ? 0x7fc00000u : 0u;
    }
#pragma unroll
    for (int j = 0; j < GF; ++j) pp[tid * GF + j] = __uint_as_float(v[j]);
    pp[GH * GF + tid] = ok ? gb : __int_as_float(0x7fc00000);
  }
  if (!ok) tc_wait(&mbar, (iter - 1) & 1);  // a late commit: wait again (bounded) before freeing
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem));
}

// ---------------------------------------------------------------------
// decoder: y = Wd h + bd;  inference: z_out = z + s_z y
// training: dy = 2 s_z (z + s_z y - delta) / |delta|^2, dh = Wd^T dy,
// loss and dWd / dbd partials per block
// ---------------------------------------------------------------------
template <int DIM>
__global__ void k_gnn_decode(int64_t n, const bf16* __restrict__ h, const float* __restrict__ Wd,
                             const float* __restrict__ bd, const double* __restrict__ scal,
                             const double* __restrict__ z, double* zout) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float y[DIM];
#pragma unroll
  for (int j = 0; j < DIM; ++j) y[j] = bd[j];
  for (int k = 0; k < GH; ++k) {
    const float hk = __bfloat162float(h[i * GH + k]);
#pragma unroll
    for (int j = 0; j < DIM; ++j) y[j] = fmaf(Wd[j * GH + k], hk, y[j]);
  }
  const double sz = scal[3];
#pragma unroll
  for (int j = 0; j < DIM; ++j) zout[j * n + i] = z[j * n + i] + sz * (double)y[j];
}

template <int DIM>
__global__ void __launch_bounds__(256)
    k_gnn_decode_bwd(int64_t n, const bf16* __restrict__ h, const float* __restrict__ Wd,
                     const float* __restrict__ bd, const double* __restrict__ scal,
                     const double* __restrict__ z, const double* __restrict__ delta, float* dh,
                     float* dy_out, float* part, int part_stride) {
  __shared__ double sl[8];
  const double sz = scal[3], den = scal[4];
  double lsum = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float y[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) y[j] = bd[j];
    for (int k = 0; k < GH; ++k) {
      const float hk = __bfloat162float(h[i * GH + k]);
#pragma unroll
      for (int j = 0; j < DIM; ++j) y[j] = fmaf(Wd[j * GH + k], hk, y[j]);
    }
    float dy[DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
      const double r = z[j * n + i] + sz * (double)y[j] - delta[j * n + i];
      lsum += r * r;
      dy[j] = (float)(2.0 * sz * r / den);
      dy_out[i * DIM + j] = dy[j];
    }
    for (int k = 0; k < GH; ++k) {
      float s = 0.f;
#pragma unroll
      for (int j = 0; j < DIM; ++j) s = fmaf(Wd[j * GH + k], dy[j], s);
      dh[i * GH + k] = s;
    }
  }
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) s += sl[wv];
    part[(int64_t)blockIdx.x * part_stride + DIM * GH + DIM] = (float)(s / den);
  }
}

// decoder weight gradients: block b sums dy (x) h over its chunk of nodes
template <int DIM>
__global__ void k_gnn_decode_wgrad(int64_t n, int64_t chunk, const bf16* __restrict__ h,
                                   const float* __restrict__ dy, float* part, int part_stride) {
  const int e = threadIdx.x;
  if (e >= DIM * GH + DIM) return;
  const int64_t lo = blockIdx.x * chunk, hi = min(n, lo + chunk);
  float s = 0.f;
  if (e < DIM * GH) {
    const int j = e / GH, k = e % GH;
    for (int64_t i = lo; i < hi; ++i) s = fmaf(dy[i * DIM + j], __bfloat162float(h[i * GH + k]), s);
  } else {
    const int j = e - DIM * GH;
    for (int64_t i = lo; i < hi; ++i) s += dy[i * DIM + j];
  }
  part[(int64_t)blockIdx.x * part_stride + e] = s;
}


// layer backward, part B: dh_in = dnext + sum_k w_ik dm_{col_ik}
__global__ void k_gnn_gather_dm(int nlf, int64_t n, const int32_t* __restrict__ col,
                                const float* __restrict__ w, const float* __restrict__ dm,
                                float* dnext) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * GH) return;
  const int64_t i = e / GH;
  const int f = (int)(e % GH);
  float s = dnext[e];
  for (int k = 0; k < nlf; ++k) {
    const int32_t j = col[i * nlf + k];
    if (j >= 0) s = fmaf(w[i * nlf + k], dm[(int64_t)j * GH + f], s);
  }
  dnext[e] = s;
}


// grad[off + e] += sum over blocks b of part[b][e] (block order), e < count
__global__ void k_gnn_reduce(int nblocks, int part_stride, int count, const float* __restrict__ part,
                             float* grad, int64_t off_w, int64_t off_b, int nw, double* loss_out,
                             int loss_slot) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < count) {
    float s = 0.f;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * part_stride + e];
    grad[e < nw ? off_w + e : off_b + (e - nw)] += s;
  }
  if (loss_out && e == 0) {
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * part_stride + loss_slot];
    loss_out[0] = s;
  }
}

__global__ void k_gnn_adam(int64_t P, float* theta, const float* grad, float* m, float* v,
                           float lr, float b1, float b2, float eps, float bc1, float bc2,
                           float scale) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = grad[i] * scale;
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
}

__global__ void k_to_bf16(int64_t count, const float* __restrict__ src, bf16* dst) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < count) dst[i] = __float2bfloat16_rn(src[i]);
}

// ---------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------
constexpr int kPartStride = GH * 2 * GH + GH;  // largest partial block (layer)

Gnn* get(hofv_ctx* c) { return static_cast<Gnn*>(c->gnn); }
bf16* hbuf(Gnn* g, int l) { return g->h + (int64_t)l * g->npad * GH; }
bf16* abuf(Gnn* g, int l) { return g->a + (int64_t)l * g->npad * GH; }

void refresh_bf16(hofv_ctx* c, Gnn* g) {
  k_to_bf16<<<(GH * GF + 255) / 256, 256, 0, c->stream>>>(GH * GF, g->theta + g->off_W0, g->W0b);
  for (int l = 0; l < GL; ++l)
    k_to_bf16<<<(GH * 2 * GH + 255) / 256, 256, 0, c->stream>>>(
        GH * 2 * GH, g->theta + g->off_W[l], g->Wb + (int64_t)l * GH * 2 * GH);
}

void free_gnn(Gnn* g) {
  for (void* p : g->allocs) cudaFree(p);
  for (double* p : g->pr) cudaFree(p);
  for (double* p : g->pd) cudaFree(p);
  for (double* p : g->pz) cudaFree(p);
  delete g;
}

int ensure(hofv_ctx* c, Gnn** out) {
  if (!c->built) return fail(c, HOFV_ESTATE, "hofv_build_stencils must come first");
  Gnn* g = get(c);
  if (g && g->n == c->nc && g->dim == c->dim) {
    *out = g;
    return 0;
  }
  if (g) free_gnn(g);
  c->gnn = nullptr;
  g = new Gnn();
  g->dim = c->dim;
  g->nlf = c->nlf;
  g->n = c->nc;
  g->ntiles = (c->nc + kTcRows - 1) / kTcRows;
  g->npad = g->ntiles * kTcRows;
  int64_t o = 0;
  g->off_W0 = o; o += GH * GF;
  g->off_b0 = o; o += GH;
  for (int l = 0; l < GL; ++l) {
    g->off_W[l] = o; o += GH * 2 * GH;
    g->off_b[l] = o; o += GH;
  }
  g->off_Wd = o; o += (int64_t)c->dim * GH;
  g->off_bd = o; o += c->dim;
  g->P = o;
  g->gblocks = 2 * c->sm_count;
  HOFV_CUDA(c, cudaFuncSetAttribute(k_gnn_layer_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kTcSmem));
  HOFV_CUDA(c, cudaFuncSetAttribute(k_gnn_layer_bwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kTcBwdSmem));
  int rc = 0;
  rc |= galloc(c, g, &g->w, g->n * g->nlf);
  rc |= galloc(c, g, &g->bnd, g->n * 2);
  rc |= galloc(c, g, &g->theta, g->P);
  rc |= galloc(c, g, &g->grad, g->P);
  rc |= galloc(c, g, &g->adam_m, g->P);
  rc |= galloc(c, g, &g->adam_v, g->P);
  rc |= galloc(c, g, &g->W0b, GH * GF);
  rc |= galloc(c, g, &g->Wb, (int64_t)GL * GH * 2 * GH);
  rc |= galloc(c, g, &g->x, g->npad * GF);
  rc |= galloc(c, g, &g->h, (int64_t)(GL + 1) * g->npad * GH);
  rc |= galloc(c, g, &g->a, (int64_t)(GL + 1) * g->npad * GH);
  rc |= galloc(c, g, &g->dh0, g->npad * GH);
  rc |= galloc(c, g, &g->dh1, g->npad * GH);
  rc |= galloc(c, g, &g->dm, g->npad * GH);
  rc |= galloc(c, g, &g->part, (int64_t)g->gblocks * kPartStride + 64);
  rc |= galloc(c, g, &g->scal, 16);
  if (rc) {
    free_gnn(g);
    return HOFV_ENOMEM;
  }
  cudaMemsetAsync(g->theta, 0, sizeof(float) * g->P, c->stream);
  cudaMemsetAsync(g->grad, 0, sizeof(float) * g->P, c->stream);
  cudaMemsetAsync(g->adam_m, 0, sizeof(float) * g->P, c->stream);
  cudaMemsetAsync(g->adam_v, 0, sizeof(float) * g->P, c->stream);
  cudaMemsetAsync(g->h, 0, sizeof(bf16) * (GL + 1) * g->npad * GH, c->stream);
  cudaMemsetAsync(g->a, 0, sizeof(bf16) * (GL + 1) * g->npad * GH, c->stream);
  cudaMemsetAsync(g->x, 0, sizeof(bf16) * g->npad * GF, c->stream);
  k_gnn_graph<<<(unsigned)((g->n + 127) / 128), 128, 0, c->stream>>>(
      g->nlf, g->n, c->nfi, c->d_aj_diag, c->d_aj_col, c->d_aj_off, c->d_cface, c->d_cf, g->w,
      g->bnd);
  HOFV_CUDA(c, cudaGetLastError());
  refresh_bf16(c, g);
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  c->gnn = g;
  *out = g;
  return 0;
}

// forward pass (activations kept for backward); decode into zout if given
int forward(hofv_ctx* c, Gnn* g, const double* v, const double* z, double* zout) {
  cudaStream_t st = c->stream;
  const int64_t nd = g->n * g->dim;
  launch_norm2(v, nd, c->d_red, c->d_count, g->scal + 0, c->red_blocks, st);
  launch_norm2(z, nd, c->d_red, c->d_count, g->scal + 1, c->red_blocks, st);
  k_gnn_scales<<<1, 1, 0, st>>>(g->scal, 1.0 / sqrt((double)nd));
  const unsigned ntc = (unsigned)((g->n + kTcRows - 1) / kTcRows);
  const unsigned neb = (unsigned)std::min<int64_t>(ntc, 4 * (int64_t)c->sm_count);
  if (g->dim == 2)
    k_gnn_encode_tc<2><<<neb, 128, 0, st>>>(g->n, g->npad, ntc, v, z, g->bnd, g->scal, g->W0b,
                                            g->theta + g->off_b0, g->x, abuf(g, 0), hbuf(g, 0));
  else
    k_gnn_encode_tc<3><<<neb, 128, 0, st>>>(g->n, g->npad, ntc, v, z, g->bnd, g->scal, g->W0b,
                                            g->theta + g->off_b0, g->x, abuf(g, 0), hbuf(g, 0));
  for (int l = 0; l < GL; ++l)
    k_gnn_layer_tc<<<ntc, 128, kTcSmem, st>>>(g->nlf, g->n, g->npad, hbuf(g, l), c->d_aj_col, g->w,
                                              g->Wb + (int64_t)l * GH * 2 * GH,
                                              g->theta + g->off_b[l], abuf(g, l + 1),
                                              hbuf(g, l + 1));
  if (zout) {
    const unsigned nb = (unsigned)((g->n + 255) / 256);
    if (g->dim == 2)
      k_gnn_decode<2><<<nb, 256, 0, st>>>(g->n, hbuf(g, GL), g->theta + g->off_Wd,
                                          g->theta + g->off_bd, g->scal, z, zout);
    else
      k_gnn_decode<3><<<nb, 256, 0, st>>>(g->n, hbuf(g, GL), g->theta + g->off_Wd,
                                          g->theta + g->off_bd, g->scal, z, zout);
  }
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

// backward of one sample (after forward); gradients added to g->grad, the
// sample's loss to scal[5]
int backward(hofv_ctx* c, Gnn* g, const double* z, const double* delta) {
  cudaStream_t st = c->stream;
  const int64_t nd = g->n * g->dim;
  launch_norm2(delta, nd, c->d_red, c->d_count, g->scal + 4, c->red_blocks, st);
  k_square<<<1, 1, 0, st>>>(g->scal + 4);
  const int gb = g->gblocks;
  const int d = g->dim;
  const int64_t chunk = (g->n + gb - 1) / gb;
  if (d == 2) {
    k_gnn_decode_bwd<2><<<gb, 256, 0, st>>>(g->n, hbuf(g, GL), g->theta + g->off_Wd,
                                            g->theta + g->off_bd, g->scal, z, delta, g->dh0,
                                            g->dm, g->part, kPartStride);
    k_gnn_decode_wgrad<2><<<gb, 256, 0, st>>>(g->n, chunk, hbuf(g, GL), g->dm, g->part,
                                              kPartStride);
  } else {
    k_gnn_decode_bwd<3><<<gb, 256, 0, st>>>(g->n, hbuf(g, GL), g->theta + g->off_Wd,
                                            g->theta + g->off_bd, g->scal, z, delta, g->dh0,
                                            g->dm, g->part, kPartStride);
    k_gnn_decode_wgrad<3><<<gb, 256, 0, st>>>(g->n, chunk, hbuf(g, GL), g->dm, g->part,
                                              kPartStride);
  }
  k_gnn_reduce<<<(d * GH + d + 255) / 256, 256, 0, st>>>(gb, kPartStride, d * GH + d, g->part,
                                                          g->grad, g->off_Wd, g->off_bd, d * GH,
                                                          g->scal + 5, d * GH + d);
  float* dcur = g->dh0;
  float* dnext = g->dh1;
  const int64_t ntc = (g->n + kTcRows - 1) / kTcRows;
  const int lbt = (int)std::min<int64_t>(ntc, gb);
  for (int l = GL - 1; l >= 0; --l) {
    k_gnn_layer_bwd_tc<<<lbt, 128, kTcBwdSmem, st>>>(
        g->nlf, g->n, ntc, hbuf(g, l), abuf(g, l + 1), c->d_aj_col, g->w,
        g->Wb + (int64_t)l * GH * 2 * GH, dcur, dnext, g->dm, g->part, kPartStride);
    k_gnn_reduce<<<(GH * 2 * GH + GH + 255) / 256, 256, 0, st>>>(
        lbt, kPartStride, GH * 2 * GH + GH, g->part, g->grad, g->off_W[l], g->off_b[l], GH * 2 * GH,
        nullptr, 0);
    k_gnn_gather_dm<<<(unsigned)((g->n * GH + 255) / 256), 256, 0, st>>>(g->nlf, g->n, c->d_aj_col,
                                                                         g->w, g->dm, dnext);
    std::swap(dcur, dnext);
  }
  k_gnn_encode_bwd_tc<<<lbt, 128, 0, st>>>(g->n, g->npad, ntc, g->x, abuf(g, 0), dcur, g->part,
                                            kPartStride);
  k_gnn_reduce<<<(GH * GF + GH + 255) / 256, 256, 0, st>>>(lbt, kPartStride, GH * GF + GH, g->part,
                                                            g->grad, g->off_W0, g->off_b0, GH * GF,
                                                            nullptr, 0);
  HOFV_CUDA(c, cudaGetLastError());
  return 0;
}

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double gauss(uint64_t& s) {
  const double u1 = ((splitmix(s) >> 11) + 1.0) * (1.0 / 9007199254740993.0);
  const double u2 = (splitmix(s) >> 11) * (1.0 / 9007199254740992.0);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

}  // namespace

int gnn_apply(hofv_ctx* c, const double* v, const double* z_aj, double* z) {
  Gnn* g = get(c);
  if (!g) return fail(c, HOFV_ESTATE, "no learned preconditioner loaded");
  return forward(c, g, v, z_aj, z);
}

void gnn_release(hofv_ctx* c) {
  if (c->gnn) free_gnn(get(c));
  c->gnn = nullptr;
}

}  // namespace hofv

using namespace hofv;

extern "C" {

int hofv_gnn_init(hofv_ctx* c, uint64_t seed, double out_scale) {
  if (!c) return HOFV_EINVAL;
  Gnn* g = nullptr;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  std::vector<float> th((size_t)g->P, 0.f);
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 12345;
  for (int i = 0; i < GH * GF; ++i) th[g->off_W0 + i] = (float)(gauss(s) * sqrt(2.0 / GF));
  for (int l = 0; l < GL; ++l)
    for (int i = 0; i < GH * 2 * GH; ++i) th[g->off_W[l] + i] = (float)(gauss(s) * sqrt(1.0 / (2 * GH)));
  for (int i = 0; i < g->dim * GH; ++i) th[g->off_Wd + i] = (float)(gauss(s) * out_scale / sqrt((double)GH));
  HOFV_CUDA(c, cudaMemcpy(g->theta, th.data(), sizeof(float) * g->P, cudaMemcpyHostToDevice));
  HOFV_CUDA(c, cudaMemset(g->adam_m, 0, sizeof(float) * g->P));
  HOFV_CUDA(c, cudaMemset(g->adam_v, 0, sizeof(float) * g->P));
  g->adam_t = 0;
  refresh_bf16(c, g);
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOFV_OK;
}

int hofv_gnn_num_params(hofv_ctx* c, int64_t* n) {
  if (!c || !n) return HOFV_EINVAL;
  Gnn* g = nullptr;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  *n = g->P;
  return HOFV_OK;
}

int hofv_gnn_get_params(hofv_ctx* c, float* host, int64_t n) {
  Gnn* g = nullptr;
  if (!c || !host) return HOFV_EINVAL;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  if (n != g->P) return fail(c, HOFV_EINVAL, "parameter count mismatch");
  HOFV_CUDA(c, cudaMemcpy(host, g->theta, sizeof(float) * n, cudaMemcpyDeviceToHost));
  return HOFV_OK;
}

int hofv_gnn_set_params(hofv_ctx* c, const float* host, int64_t n) {
  Gnn* g = nullptr;
  if (!c || !host) return HOFV_EINVAL;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  if (n != g->P) return fail(c, HOFV_EINVAL, "parameter count mismatch");
  HOFV_CUDA(c, cudaMemcpy(g->theta, host, sizeof(float) * n, cudaMemcpyHostToDevice));
  refresh_bf16(c, g);
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOFV_OK;
}

int hofv_gnn_save(hofv_ctx* c, const char* path) {
  Gnn* g = nullptr;
  if (!c || !path) return HOFV_EINVAL;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  std::vector<float> th((size_t)g->P);
  HOFV_CUDA(c, cudaMemcpy(th.data(), g->theta, sizeof(float) * g->P, cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, HOFV_EINVAL, std::string("cannot write ") + path);
  const char magic[8] = {'H', 'O', 'F', 'V', 'G', 'N', 'N', '1'};
  const int64_t hdr[3] = {g->dim, GH, g->P};
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int64_t), 3, f) == 3 &&
            fwrite(th.data(), sizeof(float), th.size(), f) == th.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? HOFV_OK : fail(c, HOFV_EINVAL, "write failed");
}

int hofv_gnn_load(hofv_ctx* c, const char* path) {
  Gnn* g = nullptr;
  if (!c || !path) return HOFV_EINVAL;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, HOFV_EINVAL, std::string("cannot read ") + path);
  char magic[8];
  int64_t hdr[3];
  std::vector<float> th((size_t)g->P);
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "HOFVGNN1", 8) == 0 &&
            fread(hdr, sizeof(int64_t), 3, f) == 3 && hdr[0] == g->dim && hdr[1] == GH &&
            hdr[2] == g->P && fread(th.data(), sizeof(float), th.size(), f) == th.size();
  fclose(f);
  if (!ok) return fail(c, HOFV_EINVAL, "not a learned-preconditioner file for this dimension");
  for (float v : th)
    if (!std::isfinite(v)) return fail(c, HOFV_ENAN, "non-finite weight in the file");
  HOFV_CUDA(c, cudaMemcpy(g->theta, th.data(), sizeof(float) * g->P, cudaMemcpyHostToDevice));
  refresh_bf16(c, g);
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOFV_OK;
}

int hofv_gnn_forward(hofv_ctx* c, const double* v, const double* z, double* zout) {
  Gnn* g = nullptr;
  if (!c || !v || !z || !zout) return HOFV_EINVAL;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  return forward(c, g, v, z, zout);
}

int hofv_gnn_loss_grad(hofv_ctx* c, const double* v, const double* z, const double* delta,
                       double* loss, float* grad_host) {
  Gnn* g = nullptr;
  if (!c || !v || !z || !delta) return HOFV_EINVAL;
  int rc = ensure(c, &g);
  if (rc) return rc;
  HOFV_CUDA(c, cudaMemsetAsync(g->grad, 0, sizeof(float) * g->P, c->stream));
  rc = forward(c, g, v, z, nullptr);
  if (rc) return rc;
  rc = backward(c, g, z, delta);
  if (rc) return rc;
  if (loss)
    HOFV_CUDA(c, cudaMemcpyAsync(loss, g->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (grad_host)
    HOFV_CUDA(c, cudaMemcpyAsync(grad_host, g->grad, sizeof(float) * g->P, cudaMemcpyDeviceToHost,
                                 c->stream));
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  return HOFV_OK;
}

int hofv_gnn_record(hofv_ctx* c, const double* r, const double* delta) {
  Gnn* g = nullptr;
  if (!c || !r || !delta) return HOFV_EINVAL;
  const int rc = ensure(c, &g);
  if (rc) return rc;
  const size_t bytes = sizeof(double) * g->n * g->dim;
  double *pr = nullptr, *pd = nullptr;
  if (cudaMalloc(&pr, bytes) != cudaSuccess) return fail(c, HOFV_ENOMEM, "training pair storage");
  if (cudaMalloc(&pd, bytes) != cudaSuccess) {
    cudaFree(pr);
    return fail(c, HOFV_ENOMEM, "training pair storage");
  }
  HOFV_CUDA(c, cudaMemcpyAsync(pr, r, bytes, cudaMemcpyDeviceToDevice, c->stream));
  HOFV_CUDA(c, cudaMemcpyAsync(pd, delta, bytes, cudaMemcpyDeviceToDevice, c->stream));
  g->pr.push_back(pr);
  g->pd.push_back(pd);
  g->pz.push_back(nullptr);
  return HOFV_OK;
}

int hofv_gnn_pairs(hofv_ctx* c, int32_t* count) {
  if (!c || !count) return HOFV_EINVAL;
  Gnn* g = get(c);
  *count = g ? (int32_t)g->pr.size() : 0;
  return HOFV_OK;
}

int hofv_gnn_clear_pairs(hofv_ctx* c) {
  if (!c) return HOFV_EINVAL;
  Gnn* g = get(c);
  if (!g) return HOFV_OK;
  cudaStreamSynchronize(c->stream);
  for (double* p : g->pr) cudaFree(p);
  for (double* p : g->pd) cudaFree(p);
  for (double* p : g->pz) cudaFree(p);
  g->pr.clear();
  g->pd.clear();
  g->pz.clear();
  return HOFV_OK;
}

int hofv_gnn_train(hofv_ctx* c, const hofv_train_opts* opts, hofv_train_stats* stats) {
  Gnn* g = nullptr;
  if (!c || !opts) return HOFV_EINVAL;
  int rc = ensure(c, &g);
  if (rc) return rc;
  if (!c->have_mat) return fail(c, HOFV_ESTATE, "hofv_set_material must come first");
  const int np = (int)g->pr.size();
  if (np == 0) return fail(c, HOFV_ESTATE, "no recorded training pairs");
  if (opts->epochs < 1 || opts->batch < 1 || !(opts->lr > 0)) return fail(c, HOFV_EINVAL, "bad training options");
  const auto t0 = std::chrono::steady_clock::now();
  const size_t bytes = sizeof(double) * g->n * g->dim;
  // preconditioned inputs z = P_AJ^{-1} r, computed once per pair
  for (int p = 0; p < np; ++p) {
    if (g->pz[p]) continue;
    if (cudaMalloc(&g->pz[p], bytes) != cudaSuccess) return fail(c, HOFV_ENOMEM, "training storage");
    rc = aj_precondition(c, HOFV_PC_AJ32, opts->inner_iters, g->pr[p], g->pz[p]);
    if (rc) return rc;
  }
  std::vector<int> order(np);
  for (int i = 0; i < np; ++i) order[i] = i;
  uint64_t s = opts->seed + 7;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  double first = -1.0, last = 0.0;
  int in_batch = 0;
  HOFV_CUDA(c, cudaMemsetAsync(g->grad, 0, sizeof(float) * g->P, c->stream));
  for (int ep = 0; ep < opts->epochs; ++ep) {
    for (int i = np - 1; i > 0; --i) std::swap(order[i], order[splitmix(s) % (uint64_t)(i + 1)]);
    double ep_loss = 0.0;
    for (int k = 0; k < np; ++k) {
      const int p = order[k];
      rc = forward(c, g, g->pr[p], g->pz[p], nullptr);
      if (rc) return rc;
      rc = backward(c, g, g->pz[p], g->pd[p]);
      if (rc) return rc;
      double L = 0.0;
      HOFV_CUDA(c, cudaMemcpyAsync(&L, g->scal + 5, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
      if (!std::isfinite(L)) return fail(c, HOFV_ENAN, "non-finite training loss");
      ep_loss += L;
      if (++in_batch == opts->batch || k == np - 1) {
        g->adam_t++;
        const float bc1 = 1.f - powf(b1, (float)g->adam_t), bc2 = 1.f - powf(b2, (float)g->adam_t);
        k_gnn_adam<<<(unsigned)((g->P + 255) / 256), 256, 0, c->stream>>>(
            g->P, g->theta, g->grad, g->adam_m, g->adam_v, (float)opts->lr, b1, b2, eps, bc1, bc2,
            1.f / in_batch);
        refresh_bf16(c, g);
        HOFV_CUDA(c, cudaMemsetAsync(g->grad, 0, sizeof(float) * g->P, c->stream));
        in_batch = 0;
      }
    }
    ep_loss /= np;
    if (first < 0) first = ep_loss;
    last = ep_loss;
    if (opts->verbose) fprintf(stderr, "[hofv] gnn epoch %d loss %.6f\n", ep, ep_loss);
  }
  HOFV_CUDA(c, cudaStreamSynchronize(c->stream));
  if (stats) {
    stats->pairs = np;
    stats->epochs = opts->epochs;
    stats->loss_first = first;
    stats->loss_last = last;
    stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return HOFV_OK;
}

}  // extern "C"
