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
// Node-wise GEMMs run on the tensor cores (mma.sync m16n8k16, BF16 inputs,
// FP32 accumulation) from padded shared-memory tiles of 64 nodes; the
// message passing is a gather over the symmetric graph, so its transpose in
// the backward pass is the same gather (no atomics); weight gradients are
// accumulated per block and reduced in block order (deterministic).
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
constexpr int GT = 64;          // nodes per tile
constexpr int GTHREADS = 128;   // 4 warps, 16 nodes each
constexpr int kLayerBwdSmem = (int)sizeof(__nv_bfloat16) *
                              (64 * (2 * 64 + 8) + 2 * 64 * (64 + 8) + 64 * (64 + 8) +
                               64 * (64 + 8) + 2 * 64 * (64 + 8));
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

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// A: row-major [rows][lda] bf16 in smem; fragment of rows row0..row0+15, cols k0..k0+15
__device__ __forceinline__ void frag_a(uint32_t* a, const bf16* A, int lda, int row0, int k0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  a[0] = *reinterpret_cast<const uint32_t*>(A + (row0 + g) * lda + k0 + 2 * t);
  a[1] = *reinterpret_cast<const uint32_t*>(A + (row0 + g + 8) * lda + k0 + 2 * t);
  a[2] = *reinterpret_cast<const uint32_t*>(A + (row0 + g) * lda + k0 + 2 * t + 8);
  a[3] = *reinterpret_cast<const uint32_t*>(A + (row0 + g + 8) * lda + k0 + 2 * t + 8);
}
// B given as BT: row-major [N][ldb] bf16 (row n holds column n of B over k)
__device__ __forceinline__ void frag_b(uint32_t* b, const bf16* BT, int ldb, int n0, int k0, int lane) {
  const int g = lane >> 2, t = lane & 3;
  b[0] = *reinterpret_cast<const uint32_t*>(BT + (n0 + g) * ldb + k0 + 2 * t);
  b[1] = *reinterpret_cast<const uint32_t*>(BT + (n0 + g) * ldb + k0 + 2 * t + 8);
}

__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// ---------------------------------------------------------------------
// graph: symmetric weights and boundary fractions
// ---------------------------------------------------------------------
__global__ void k_gnn_graph(int nlf, int64_t n, int64_t nfi, const double* __restrict__ diag,
                            const int32_t* __restrict__ col, const double* __restrict__ off,
                            const int32_t* __restrict__ cface, float* w, float* bnd) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int nd = 0, nt = 0;
  for (int k = 0; k < nlf; ++k) {
    const int32_t j = col[i * nlf + k];
    w[i * nlf + k] = j >= 0 ? (float)(off[i * nlf + k] / sqrt(diag[i] * diag[j])) : 0.f;
    const int32_t code = cface[i * nlf + k];
    if (code == 0) ++nt;
    else if (code > 0 && code - 1 >= nfi) ++nd;
  }
  bnd[2 * i] = (float)nd / nlf;
  bnd[2 * i + 1] = (float)nt / nlf;
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
// encoder: x (built from v, z) -> h0 = relu(W0 x + b0)
// ---------------------------------------------------------------------
template <int DIM>
__global__ void __launch_bounds__(GTHREADS)
    k_gnn_encode(int64_t n, const double* __restrict__ v, const double* __restrict__ z,
                 const float* __restrict__ bnd, const double* __restrict__ scal,
                 const bf16* __restrict__ W0b, const float* __restrict__ b0, bf16* xg, bf16* a0,
                 bf16* h0) {
  __shared__ __align__(16) bf16 sx[GT][GF + 8];
  __shared__ __align__(16) bf16 sw[GH][GF + 8];
  const int64_t base = (int64_t)blockIdx.x * GT;
  const double isv = 1.0 / scal[2], isz = 1.0 / scal[3];
  for (int e = threadIdx.x; e < GT * GF; e += GTHREADS) {
    const int r = e / GF, f = e % GF;
    const int64_t i = base + r;
    float val = 0.f;
    if (i < n) {
      if (f < DIM) val = (float)(v[f * n + i] * isv);
      else if (f < 2 * DIM) val = (float)(z[(f - DIM) * n + i] * isz);
      else if (f < 2 * DIM + 2) val = bnd[2 * i + (f - 2 * DIM)];
    }
    const bf16 bv = __float2bfloat16_rn(val);
    sx[r][f] = bv;
    xg[(base + r) * GF + f] = bv;
  }
  for (int e = threadIdx.x; e < GH * GF; e += GTHREADS) sw[e / GF][e % GF] = W0b[e];
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  uint32_t af[4];
  frag_a(af, &sx[0][0], GF + 8, wp * 16, 0, lane);
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < GH / 8; ++nt) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    uint32_t bfr[2];
    frag_b(bfr, &sw[0][0], GF + 8, nt * 8, 0, lane);
    mma16816(acc, af, bfr);
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int64_t row = base + wp * 16 + g + 8 * hh;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int colm = nt * 8 + 2 * t + cc;
        const float pre = acc[2 * hh + cc] + b0[colm];
        a0[row * GH + colm] = __float2bfloat16_rn(pre);
        h0[row * GH + colm] = __float2bfloat16_rn(relu(pre));
      }
    }
  }
}

// gather m_i = sum_k w_ik h_{col_ik} for the tile into smem (bf16), plus the
// tile's own h, as the 64 x 128 operand [h | m]
__device__ __forceinline__ void load_hm_tile(int nlf, int64_t n, int64_t base,
                                             const bf16* __restrict__ h,
                                             const int32_t* __restrict__ col,
                                             const float* __restrict__ w, bf16 (*sX)[2 * GH + 8]) {
  for (int e = threadIdx.x; e < GT * (GH / 8); e += GTHREADS) {
    const int r = e / (GH / 8), ch = e % (GH / 8);
    const int64_t i = base + r;
    float mv[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint4 own = make_uint4(0, 0, 0, 0);
    if (i < n) {
      own = *reinterpret_cast<const uint4*>(h + i * GH + ch * 8);
      for (int k = 0; k < nlf; ++k) {
        const int32_t j = col[i * nlf + k];
        if (j < 0) continue;
        const float wk = w[i * nlf + k];
        const uint4 hv = *reinterpret_cast<const uint4*>(h + (int64_t)j * GH + ch * 8);
        const bf16* hb = reinterpret_cast<const bf16*>(&hv);
#pragma unroll
        for (int q = 0; q < 8; ++q) mv[q] = fmaf(wk, __bfloat162float(hb[q]), mv[q]);
      }
    }
    *reinterpret_cast<uint4*>(&sX[r][ch * 8]) = own;
#pragma unroll
    for (int q = 0; q < 8; ++q) sX[r][GH + ch * 8 + q] = __float2bfloat16_rn(mv[q]);
  }
}

// ---------------------------------------------------------------------
// one message-passing layer: h_out = h_in + relu(W [h_in; m] + b)
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(GTHREADS)
    k_gnn_layer(int nlf, int64_t n, const bf16* __restrict__ hin, const int32_t* __restrict__ col,
                const float* __restrict__ w, const bf16* __restrict__ Wb,
                const float* __restrict__ b, bf16* aout, bf16* hout) {
  __shared__ __align__(16) bf16 sX[GT][2 * GH + 8];
  __shared__ __align__(16) bf16 sW[GH][2 * GH + 8];
  const int64_t base = (int64_t)blockIdx.x * GT;
  load_hm_tile(nlf, n, base, hin, col, w, sX);
  for (int e = threadIdx.x; e < GH * 2 * GH / 8; e += GTHREADS) {
    const int r = e / (2 * GH / 8), ch = e % (2 * GH / 8);
    *reinterpret_cast<uint4*>(&sW[r][ch * 8]) = *reinterpret_cast<const uint4*>(Wb + r * 2 * GH + ch * 8);
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float acc[GH / 8][4];
#pragma unroll
  for (int nt = 0; nt < GH / 8; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < 2 * GH / 16; ++kk) {
    uint32_t af[4];
    frag_a(af, &sX[0][0], 2 * GH + 8, wp * 16, kk * 16, lane);
#pragma unroll
    for (int nt = 0; nt < GH / 8; ++nt) {
      uint32_t bfr[2];
      frag_b(bfr, &sW[0][0], 2 * GH + 8, nt * 8, kk * 16, lane);
      mma16816(acc[nt], af, bfr);
    }
  }
#pragma unroll
  for (int nt = 0; nt < GH / 8; ++nt)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int r = wp * 16 + g + 8 * hh;
      const int64_t row = base + r;
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int colm = nt * 8 + 2 * t + cc;
        const float pre = acc[nt][2 * hh + cc] + b[colm];
        aout[row * GH + colm] = __float2bfloat16_rn(pre);
        hout[row * GH + colm] = __float2bfloat16_rn(__bfloat162float(sX[r][colm]) + relu(pre));
      }
    }
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

// ---------------------------------------------------------------------
// layer backward, part A (persistent over tiles):
//   dpre = dh_out * (a > 0)
//   [dself | dm] = dpre W          -> dnext = dh_out + dself,  dm
//   dW += dpre^T [h_in | m],  db += sum dpre   (block partials)
// ---------------------------------------------------------------------
__global__ void __launch_bounds__(GTHREADS)
    k_gnn_layer_bwd(int nlf, int64_t n, int64_t ntiles, const bf16* __restrict__ hin,
                    const bf16* __restrict__ a, const int32_t* __restrict__ col,
                    const float* __restrict__ w, const bf16* __restrict__ Wb,
                    const float* __restrict__ dh_out, float* dnext, float* dm, float* part,
                    int part_stride) {
  // dynamic shared memory (kLayerBwdSmem bytes):
  //   sX  [GT][2GH+8]   [h | m], rows = nodes
  //   sXT [2GH][GT+8]   transposed, rows = features
  //   sD  [GT][GH+8]    dpre, rows = nodes
  //   sDT [GH][GT+8]    dpre^T, rows = output features
  //   sWT [2GH][GH+8]   W^T, rows = input features
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 (*sX)[2 * GH + 8] = reinterpret_cast<bf16 (*)[2 * GH + 8]>(smem_raw);
  bf16 (*sXT)[GT + 8] = reinterpret_cast<bf16 (*)[GT + 8]>(&sX[GT][0]);
  bf16 (*sD)[GH + 8] = reinterpret_cast<bf16 (*)[GH + 8]>(&sXT[2 * GH][0]);
  bf16 (*sDT)[GT + 8] = reinterpret_cast<bf16 (*)[GT + 8]>(&sD[GT][0]);
  bf16 (*sWT)[GH + 8] = reinterpret_cast<bf16 (*)[GH + 8]>(&sDT[GH][0]);
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  for (int e = threadIdx.x; e < GH * 2 * GH; e += GTHREADS) {
    const int o = e / (2 * GH), i = e % (2 * GH);
    sWT[i][o] = Wb[e];
  }
  float gw[2 * GH / 8][4];  // this warp's 16 output rows x 128 inputs of dW
#pragma unroll
  for (int nt = 0; nt < 2 * GH / 8; ++nt) gw[nt][0] = gw[nt][1] = gw[nt][2] = gw[nt][3] = 0.f;
  float gb = 0.f;           // db for output feature threadIdx.x (< 64)
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * GT;
    __syncthreads();
    load_hm_tile(nlf, n, base, hin, col, w, sX);
    for (int e = threadIdx.x; e < GT * GH; e += GTHREADS) {
      const int r = e / GH, f = e % GH;
      const int64_t i = base + r;
      float d = 0.f;
      if (i < n && __bfloat162float(a[i * GH + f]) > 0.f) d = dh_out[i * GH + f];
      const bf16 db = __float2bfloat16_rn(d);
      sD[r][f] = db;
      sDT[f][r] = db;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < GT * 2 * GH; e += GTHREADS) {
      const int r = e / (2 * GH), f = e % (2 * GH);
      sXT[f][r] = sX[r][f];
    }
    if (threadIdx.x < GH)
      for (int r = 0; r < GT; ++r) gb += __bfloat162float(sDT[threadIdx.x][r]);
    __syncthreads();
    // [dself | dm] (16 nodes x 128 per warp) = dpre (16 x 64) x W (64 x 128)
#pragma unroll
    for (int nt = 0; nt < 2 * GH / 8; ++nt) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kk = 0; kk < GH / 16; ++kk) {
        uint32_t af[4], bfr[2];
        frag_a(af, &sD[0][0], GH + 8, wp * 16, kk * 16, lane);
        frag_b(bfr, &sWT[0][0], GH + 8, nt * 8, kk * 16, lane);
        mma16816(acc, af, bfr);
      }
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int64_t i = base + wp * 16 + g + 8 * hh;
        if (i >= n) continue;
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int colm = nt * 8 + 2 * t + cc;
          if (colm < GH)
            dnext[i * GH + colm] = dh_out[i * GH + colm] + acc[2 * hh + cc];
          else
            dm[i * GH + colm - GH] = acc[2 * hh + cc];
        }
      }
    }
    // dW (16 out rows x 128 per warp) += dpre^T (16 x 64 nodes) x X (64 nodes x 128)
#pragma unroll
    for (int kk = 0; kk < GT / 16; ++kk) {
      uint32_t af[4];
      frag_a(af, &sDT[0][0], GT + 8, wp * 16, kk * 16, lane);
#pragma unroll
      for (int nt = 0; nt < 2 * GH / 8; ++nt) {
        uint32_t bfr[2];
        frag_b(bfr, &sXT[0][0], GT + 8, nt * 8, kk * 16, lane);
        mma16816(gw[nt], af, bfr);
      }
    }
  }
  float* pp = part + (int64_t)blockIdx.x * part_stride;
#pragma unroll
  for (int nt = 0; nt < 2 * GH / 8; ++nt)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int o = wp * 16 + g + 8 * hh, i = nt * 8 + 2 * t + cc;
        pp[o * 2 * GH + i] = gw[nt][2 * hh + cc];
      }
  if (threadIdx.x < GH) pp[GH * 2 * GH + threadIdx.x] = gb;
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

// encoder backward (persistent): dpre0 = dh0 * (a0 > 0); dW0 += dpre0^T x
__global__ void __launch_bounds__(GTHREADS)
    k_gnn_encode_bwd(int64_t n, int64_t ntiles, const bf16* __restrict__ xg,
                     const bf16* __restrict__ a0, const float* __restrict__ dh, float* part,
                     int part_stride) {
  __shared__ __align__(16) bf16 sDT[GH][GT + 8];
  __shared__ __align__(16) bf16 sXT[GF][GT + 8];
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  float gw[GF / 8][4];
#pragma unroll
  for (int nt = 0; nt < GF / 8; ++nt) gw[nt][0] = gw[nt][1] = gw[nt][2] = gw[nt][3] = 0.f;
  float gb = 0.f;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t base = tile * GT;
    __syncthreads();
    for (int e = threadIdx.x; e < GT * GH; e += GTHREADS) {
      const int r = e / GH, f = e % GH;
      const int64_t i = base + r;
      float d = 0.f;
      if (i < n && __bfloat162float(a0[i * GH + f]) > 0.f) d = dh[i * GH + f];
      sDT[f][r] = __float2bfloat16_rn(d);
    }
    for (int e = threadIdx.x; e < GT * GF; e += GTHREADS) {
      const int r = e / GF, f = e % GF;
      sXT[f][r] = xg[(base + r) * GF + f];
    }
    __syncthreads();
    if (threadIdx.x < GH)
      for (int r = 0; r < GT; ++r) gb += __bfloat162float(sDT[threadIdx.x][r]);
#pragma unroll
    for (int kk = 0; kk < GT / 16; ++kk) {
      uint32_t af[4];
      frag_a(af, &sDT[0][0], GT + 8, wp * 16, kk * 16, lane);
#pragma unroll
      for (int nt = 0; nt < GF / 8; ++nt) {
        uint32_t bfr[2];
        frag_b(bfr, &sXT[0][0], GT + 8, nt * 8, kk * 16, lane);
        mma16816(gw[nt], af, bfr);
      }
    }
  }
  float* pp = part + (int64_t)blockIdx.x * part_stride;
#pragma unroll
  for (int nt = 0; nt < GF / 8; ++nt)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh)
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int o = wp * 16 + g + 8 * hh, i = nt * 8 + 2 * t + cc;
        pp[o * GF + i] = gw[nt][2 * hh + cc];
      }
  if (threadIdx.x < GH) pp[GH * GF + threadIdx.x] = gb;
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
  g->ntiles = (c->nc + GT - 1) / GT;
  g->npad = g->ntiles * GT;
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
  HOFV_CUDA(c, cudaFuncSetAttribute(k_gnn_layer_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    kLayerBwdSmem));
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
      g->nlf, g->n, c->nfi, c->d_aj_diag, c->d_aj_col, c->d_aj_off, c->d_cface, g->w, g->bnd);
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
  const unsigned nt = (unsigned)g->ntiles;
  if (g->dim == 2)
    k_gnn_encode<2><<<nt, GTHREADS, 0, st>>>(g->n, v, z, g->bnd, g->scal, g->W0b,
                                             g->theta + g->off_b0, g->x, abuf(g, 0), hbuf(g, 0));
  else
    k_gnn_encode<3><<<nt, GTHREADS, 0, st>>>(g->n, v, z, g->bnd, g->scal, g->W0b,
                                             g->theta + g->off_b0, g->x, abuf(g, 0), hbuf(g, 0));
  for (int l = 0; l < GL; ++l)
    k_gnn_layer<<<nt, GTHREADS, 0, st>>>(g->nlf, g->n, hbuf(g, l), c->d_aj_col, g->w,
                                         g->Wb + (int64_t)l * GH * 2 * GH, g->theta + g->off_b[l],
                                         abuf(g, l + 1), hbuf(g, l + 1));
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
  const int lb = (int)std::min<int64_t>(g->ntiles, gb);
  for (int l = GL - 1; l >= 0; --l) {
    k_gnn_layer_bwd<<<lb, GTHREADS, kLayerBwdSmem, st>>>(g->nlf, g->n, g->ntiles, hbuf(g, l), abuf(g, l + 1),
                                             c->d_aj_col, g->w, g->Wb + (int64_t)l * GH * 2 * GH,
                                             dcur, dnext, g->dm, g->part, kPartStride);
    k_gnn_reduce<<<(GH * 2 * GH + GH + 255) / 256, 256, 0, st>>>(
        lb, kPartStride, GH * 2 * GH + GH, g->part, g->grad, g->off_W[l], g->off_b[l], GH * 2 * GH,
        nullptr, 0);
    k_gnn_gather_dm<<<(unsigned)((g->n * GH + 255) / 256), 256, 0, st>>>(g->nlf, g->n, c->d_aj_col,
                                                                         g->w, g->dm, dnext);
    std::swap(dcur, dnext);
  }
  k_gnn_encode_bwd<<<lb, GTHREADS, 0, st>>>(g->n, g->ntiles, g->x, abuf(g, 0), dcur, g->part,
                                            kPartStride);
  k_gnn_reduce<<<(GH * GF + GH + 255) / 256, 256, 0, st>>>(lb, kPartStride, GH * GF + GH, g->part,
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
