// Surrogate MLP of the min-power objective over the transmitter position:
// Fourier features (32 frequencies: sin and cos of 2 pi B_j . x), four
// Linear(256) + SiLU layers and Linear(1); BF16 weights and activations, FP32
// accumulation, FP32 master weights trained with Adam.
//
// The dense layers are one GEMM kernel C = A . Bt^T (both operands stored
// K-contiguous) on the tensor cores (mma.sync m16n8k16 BF16 -> FP32, operands
// staged in shared memory and fed by ldmatrix), with three epilogues:
//   FWD: z = acc + bias; store z (FP32), h = SiLU(z) as BF16 row-major and
//        transposed (the transposed copy is the B operand of the weight gradient);
//   DH:  the GEMM is dH = dZ . W; store dZ_prev = dH * SiLU'(z_prev) (BF16, both layouts);
//   DW:  the GEMM is dW = dZ^T . H (K = batch); store FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <mutex>
#include <utility>

#include "drt.h"
#include "drt_internal.h"

namespace drt {
namespace mlp {

constexpr int NFREQ = DRT_MLP_FREQS;
constexpr int NFEAT = 2 * DRT_MLP_FREQS;
constexpr int WID = DRT_MLP_WIDTH;
constexpr int NL = DRT_MLP_LAYERS;

typedef __nv_bfloat16 bf16;

// Offsets (in floats) of each parameter block in the flat FP32 vector, and
// (in bf16 elements) of the shadow copies.
struct Layout {
  long long w[NL], b[NL], w5, b5, total;
  long long sw[NL], swt[NL], sw5, stotal;
  long long swc[NL];   // W_l in 256 x 32 K-chunks, each in the tensor-core smem layout
  int k[NL];
};

// K-chunk width of the chunked weight copy, and the byte offset of element
// (n, k) of a [256 x 32] chunk in the canonical no-swizzle K-major layout of the
// tcgen05 operands (8-row x 16-byte core matrices, four along K per 8-row group).
constexpr int WCHUNK_K = 32;
__host__ __device__ constexpr unsigned chunk_woff(int n, int k) {
  return (unsigned)((((n >> 3) * (WCHUNK_K / 8) + (k >> 3)) << 7) + ((n & 7) << 4) + ((k & 7) << 1));
}

__host__ __device__ inline Layout layout() {
  Layout L{};
  long long o = 0, so = 0;
  for (int l = 0; l < NL; ++l) {
    L.k[l] = (l == 0) ? NFEAT : WID;
    L.w[l] = o;
    o += (long long)WID * L.k[l];
    L.b[l] = o;
    o += WID;
    L.sw[l] = so;
    so += (long long)WID * L.k[l];
    L.swt[l] = so;
    so += (long long)WID * L.k[l];
  }
  L.w5 = o;
  o += WID;
  L.b5 = o;
  o += 1;
  L.total = o;
  L.sw5 = so;
  so += WID;
  for (int l = 0; l < NL; ++l) {
    L.swc[l] = so;
    so += (long long)WID * L.k[l];
  }
  L.stotal = so;
  return L;
}

enum : int { EPI_FWD = 0, EPI_DH = 1, EPI_DW = 2 };

struct GemmArgs {
  const bf16* A;
  int lda;
  const bf16* Bt;
  int ldb;
  int M, N, K;
  const float* bias;   // FWD
  float* Z;            // FWD: out [M][ldz]; DH: in (pre-activation of the layer below)
  int ldz;
  bf16* H;             // FWD: SiLU(z); DH: dZ  [M][ldh]
  int ldh;
  bf16* HT;            // transposed copy [N][ldht] (optional)
  int ldht;
  float* C;            // DW: out [M][ldc]; with split-K, partial z at C + z * M * ldc
  int ldc;
  int k_splits;        // DW: K is split into k_splits equal slices (blockIdx.z), >= 1
};

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* smem_ptr) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem_ptr);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }

// C[M x N] = A[M x K] . Bt[N x K]^T; M, N multiples of 64, K a multiple of 32.
template <int EPI>
__global__ void __launch_bounds__(128) gemm_nt_kernel(const GemmArgs g) {
  constexpr int LDS = 40;   // padded row (bf16): 80 bytes, conflict-free ldmatrix
  __shared__ __align__(16) bf16 As[64][LDS];
  __shared__ __align__(16) bf16 Bs[64][LDS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 1, wn = warp & 1;
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

  const int kz = g.K / (g.k_splits > 0 ? g.k_splits : 1);
  const int kbeg = blockIdx.z * kz, kend = kbeg + kz;
  float* C = g.C ? g.C + (size_t)blockIdx.z * g.M * g.ldc : nullptr;
  for (int k0 = kbeg; k0 < kend; k0 += 32) {
    for (int i = tid; i < 256; i += 128) {
      const int r = i >> 2, c = (i & 3) * 8;
      *reinterpret_cast<uint4*>(&As[r][c]) =
          *reinterpret_cast<const uint4*>(g.A + (size_t)(m0 + r) * g.lda + k0 + c);
      *reinterpret_cast<uint4*>(&Bs[r][c]) =
          *reinterpret_cast<const uint4*>(g.Bt + (size_t)(n0 + r) * g.ldb + k0 + c);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) ldsm_x4(a[i], &As[wm * 32 + i * 16 + (lane % 16)][kk + (lane / 16) * 8]);
#pragma unroll
      for (int jj = 0; jj < 2; ++jj) {
        uint32_t r[4];
        ldsm_x4(r, &Bs[wn * 32 + jj * 16 + (lane % 8) + (lane / 16) * 8][kk + ((lane / 8) % 2) * 8]);
        b[2 * jj][0] = r[0];
        b[2 * jj][1] = r[1];
        b[2 * jj + 1][0] = r[2];
        b[2 * jj + 1][1] = r[3];
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  const int gq = lane >> 2, tq = lane & 3;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int row = m0 + wm * 32 + i * 16 + gq + (q >> 1) * 8;
        const int col = n0 + wn * 32 + j * 8 + 2 * tq + (q & 1);
        const float v = acc[i][j][q];
        if (EPI == EPI_FWD) {
          const float z = v + g.bias[col];
          if (g.Z) g.Z[(size_t)row * g.ldz + col] = z;
          const bf16 h = __float2bfloat16(z * sigm(z));
          g.H[(size_t)row * g.ldh + col] = h;
          if (g.HT) g.HT[(size_t)col * g.ldht + row] = h;
        } else if (EPI == EPI_DH) {
          const float zp = g.Z[(size_t)row * g.ldz + col];
          const float s = sigm(zp);
          const bf16 dz = __float2bfloat16(v * s * (1.f + zp * (1.f - s)));
          g.H[(size_t)row * g.ldh + col] = dz;
          g.HT[(size_t)col * g.ldht + row] = dz;
        } else {
          C[(size_t)row * g.ldc + col] = v;
        }
      }
}

// out[i] = sum_z part[z][i] over the K splits, in split order
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, long long n,
                                     float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int z = 0; z < splits; ++z) s += part[(size_t)z * n + i];
    out[i] = s;
  }
}

// F[b] = (sin(2 pi B_j . x_b))_j, (cos(2 pi B_j . x_b))_j as BF16, row-major and transposed.
__global__ void fourier_kernel(const float* __restrict__ freqs, const float* __restrict__ x, int B,
                               bf16* __restrict__ F, bf16* __restrict__ FT) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * NFREQ; i += gridDim.x * blockDim.x) {
    const int b = i / NFREQ, j = i % NFREQ;
    const float v = 2.f * fmaf(freqs[2 * j], x[2 * b], freqs[2 * j + 1] * x[2 * b + 1]);
    float sv, cv;
    sincospif(v, &sv, &cv);
    const bf16 s = __float2bfloat16(sv), c = __float2bfloat16(cv);
    F[(size_t)b * NFEAT + j] = s;
    F[(size_t)b * NFEAT + NFREQ + j] = c;
    if (FT) {
      FT[(size_t)j * B + b] = s;
      FT[(size_t)(NFREQ + j) * B + b] = c;
    }
  }
}

// y[b] = h4[b] . w5 + b5 (one warp per row); with a target, dy[b] = 2 (y[b] - t[b]) / B.
__global__ void out_layer_kernel(const bf16* __restrict__ H4, const bf16* __restrict__ w5,
                                 const float* __restrict__ params, long long off_b5, int B,
                                 const float* __restrict__ target, float* __restrict__ y,
                                 float* __restrict__ dy) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long b = gw; b < B; b += nw) {
    float s = 0.f;
    for (int k = lane; k < WID; k += 32)
      s = fmaf(__bfloat162float(H4[b * WID + k]), __bfloat162float(w5[k]), s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
      const float yb = s + params[off_b5];
      y[b] = yb;
      if (target) dy[b] = 2.f * (yb - target[b]) / (float)B;
    }
  }
}

// loss = mean (y - t)^2 and d loss / d b5 = sum dy, in a fixed order (one block).
__global__ void __launch_bounds__(1024) loss_reduce_kernel(const float* __restrict__ y,
                                                           const float* __restrict__ t,
                                                           const float* __restrict__ dy, int B,
                                                           float* __restrict__ loss,
                                                           float* __restrict__ grad_b5) {
  __shared__ float s1[1024], s2[1024];
  float a = 0.f, c = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float d = y[b] - t[b];
    a = fmaf(d, d, a);
    c += dy[b];
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    loss[0] = s1[0] / (float)B;
    grad_b5[0] = s2[0];
  }
}

// dZ4[b][k] = dy[b] w5[k] SiLU'(z4[b][k]) (BF16, both layouts)
__global__ void out_backward_kernel(const float* __restrict__ dy, const bf16* __restrict__ w5,
                                    const float* __restrict__ Z4, int B, bf16* __restrict__ dZ,
                                    bf16* __restrict__ dZT) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)B * WID;
       i += (long long)gridDim.x * blockDim.x) {
    const long long b = i / WID;
    const int k = (int)(i % WID);
    const float z = Z4[i];
    const float s = sigm(z);
    const bf16 d = __float2bfloat16(dy[b] * __bfloat162float(w5[k]) * s * (1.f + z * (1.f - s)));
    dZ[i] = d;
    dZT[(size_t)k * B + b] = d;
  }
}

// out[r] = sum_c X[r][c] (* wvec[c]); one warp per row, fixed order.
__global__ void row_sum_kernel(const bf16* __restrict__ X, int rows, int cols,
                               const float* __restrict__ wvec, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long r = gw; r < rows; r += nw) {
    float s = 0.f;
    for (int c = lane; c < cols; c += 32) {
      const float v = __bfloat162float(X[r * cols + c]);
      s = wvec ? fmaf(v, wvec[c], s) : s + v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[r] = s;
  }
}

// Adam on the FP32 master vector; refreshes the BF16 shadows (W, W^T, w5).
// BF16 copies of parameter i (value v) in the shadow: W_l row-major, its
// transpose, its K-chunked tensor-core layout, and w5.
__device__ __forceinline__ void write_shadow(const Layout& L, bf16* __restrict__ shadow, long long i,
                                             float v) {
  for (int l = 0; l < NL; ++l) {
    const long long n_w = (long long)WID * L.k[l];
    if (i >= L.w[l] && i < L.w[l] + n_w) {
      const long long e = i - L.w[l];
      const int n = (int)(e / L.k[l]), k = (int)(e % L.k[l]);
      const bf16 b = __float2bfloat16(v);
      shadow[L.sw[l] + e] = b;
      shadow[L.swt[l] + (long long)k * WID + n] = b;
      shadow[L.swc[l] + (long long)(k / WCHUNK_K) * WID * WCHUNK_K +
             chunk_woff(n, k % WCHUNK_K) / 2] = b;
    }
  }
  if (i >= L.w5 && i < L.w5 + WID) shadow[L.sw5 + (i - L.w5)] = __float2bfloat16(v);
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, const int32_t* __restrict__ step, float lr,
                            float b1, float b2, float eps, bf16* __restrict__ shadow) {
  const Layout L = layout();
  const int t = *step + 1;
  const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.total;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (shadow) write_shadow(L, shadow, i, pi);
  }
}

__global__ void shadow_kernel(const float* __restrict__ p, bf16* __restrict__ shadow) {
  const Layout L = layout();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < L.total;
       i += (long long)gridDim.x * blockDim.x)
    write_shadow(L, shadow, i, p[i]);
}

__global__ void increment_kernel(int32_t* step) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *step += 1;
}

}  // namespace mlp
}  // namespace drt

#include "drt_mlp_tc.cuh"
#include "drt_mlp_fused.cuh"

namespace drt {
namespace mlp {

// timeout flag of the tcgen05 kernels (device-global; read and cleared by drt_mlp_tc_status)
__device__ int g_tc_status;

}  // namespace mlp

// ------------------------------------------------------------------ host side
namespace {

using mlp::bf16;

struct MlpWs {
  bf16 *F, *FT, *H[DRT_MLP_LAYERS + 1], *HT[DRT_MLP_LAYERS + 1], *dZa, *dZTa, *dZb, *dZTb;
  float *Z[DRT_MLP_LAYERS], *y, *dy, *part;
  int splits;
  size_t bytes;
};

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

MlpWs carve(void* base, int B) {
  MlpWs w{};
  char* p = static_cast<char*>(base);
  size_t o = 0;
  auto take = [&](size_t n) {
    char* r = p ? p + o : nullptr;
    o = al256(o + n);
    return r;
  };
  const size_t hb = (size_t)B * mlp::WID * sizeof(bf16);
  w.F = reinterpret_cast<bf16*>(take((size_t)B * mlp::NFEAT * sizeof(bf16)));
  w.FT = reinterpret_cast<bf16*>(take((size_t)B * mlp::NFEAT * sizeof(bf16)));
  w.H[0] = w.F;
  w.HT[0] = w.FT;
  for (int l = 1; l <= mlp::NL; ++l) {
    w.H[l] = reinterpret_cast<bf16*>(take(hb));
    w.HT[l] = reinterpret_cast<bf16*>(take(hb));
  }
  for (int l = 0; l < mlp::NL; ++l) w.Z[l] = reinterpret_cast<float*>(take((size_t)B * mlp::WID * 4));
  w.y = reinterpret_cast<float*>(take((size_t)B * 4));
  w.dy = reinterpret_cast<float*>(take((size_t)B * 4));
  w.dZa = reinterpret_cast<bf16*>(take(hb));
  w.dZTa = reinterpret_cast<bf16*>(take(hb));
  w.dZb = reinterpret_cast<bf16*>(take(hb));
  w.dZTb = reinterpret_cast<bf16*>(take(hb));
  // weight gradients reduce over the batch: split it into slices of >= 256 rows
  w.splits = std::max(1, std::min(32, B / 256));
  while (w.splits > 1 && (B % (w.splits * 64))) --w.splits;
  w.part = reinterpret_cast<float*>(take((size_t)w.splits * mlp::WID * mlp::WID * 4));
  w.bytes = o;
  return w;
}

// Which tensor-core path the dense layers use: 1 = tcgen05 (TMEM accumulator),
// 0 = mma.sync.  The tcgen05 path needs M a multiple of 128 and K of 64; other
// shapes take the mma.sync path.
std::atomic<int> g_tc_mode{1};
std::atomic<int> g_tc_skip_mma{0};
std::mutex g_tc_mu;
int* g_tc_status_ptr[64] = {};

// 72 KB of dynamic shared memory per CTA: the two 128 x 64 stages (or the FP32
// output tile) fit, and at most three CTAs (3 x 128 TMEM columns) share an SM.
constexpr int TC_SMEM = 72 * 1024;
static_assert(mlp::TcSmem<128>::BYTES <= TC_SMEM && mlp::TcSmem<64>::BYTES <= TC_SMEM, "smem");

int* tc_status_ptr() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(g_tc_mu);
  if (!g_tc_status_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, mlp::g_tc_status) != cudaSuccess) return nullptr;
    g_tc_status_ptr[dev] = static_cast<int*>(p);
    cudaFuncSetAttribute(mlp::tc_gemm_nt_kernel<mlp::EPI_FWD, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(mlp::tc_gemm_nt_kernel<mlp::EPI_DH, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(mlp::tc_gemm_nt_kernel<mlp::EPI_DW, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(mlp::tc_gemm_nt_kernel<mlp::EPI_FWD, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(mlp::tc_gemm_nt_kernel<mlp::EPI_DH, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(mlp::tc_gemm_nt_kernel<mlp::EPI_DW, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    cudaFuncSetAttribute(mlp::tc_mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         mlp::FZ_SMEM);
  }
  return g_tc_status_ptr[dev];
}

template <int EPI>
cudaError_t gemm(const mlp::GemmArgs& g, cudaStream_t st) {
  const bool tc_shape = (g.M % mlp::TC_BM == 0) && (g.K % mlp::TC_BK == 0) && (g.N % 64 == 0);
  // the training GEMMs take tcgen05 only in mode 2 (mode 1: the fused inference kernel)
  int* status = (g_tc_mode.load() == 2 && tc_shape) ? tc_status_ptr() : nullptr;
  if (status) {
    const int z = (EPI == mlp::EPI_DW && g.k_splits > 1) ? g.k_splits : 1;
    if (g.N % 128 == 0) {
      dim3 grid(g.N / 128, g.M / mlp::TC_BM, z);
      mlp::tc_gemm_nt_kernel<EPI, 128><<<grid, 128, TC_SMEM, st>>>(g, status, g_tc_skip_mma.load());
    } else {
      dim3 grid(g.N / 64, g.M / mlp::TC_BM, z);
      mlp::tc_gemm_nt_kernel<EPI, 64><<<grid, 128, TC_SMEM, st>>>(g, status, g_tc_skip_mma.load());
    }
    return cudaGetLastError();
  }
  dim3 grid(g.N / 64, g.M / 64, (EPI == mlp::EPI_DW && g.k_splits > 1) ? g.k_splits : 1);
  mlp::gemm_nt_kernel<EPI><<<grid, 128, 0, st>>>(g);
  return cudaGetLastError();
}

// forward through the hidden layers; with_train keeps Z and the transposed copies
cudaError_t mlp_hidden_forward(const float* params, const bf16* shadow, const float* freqs,
                               const float* x, int B, const MlpWs& w, bool with_train,
                               cudaStream_t st) {
  const mlp::Layout L = mlp::layout();
  const int blocks = std::min(4096, (B * mlp::NFREQ + 255) / 256);
  mlp::fourier_kernel<<<blocks, 256, 0, st>>>(freqs, x, B, w.F, with_train ? w.FT : nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int l = 0; l < mlp::NL; ++l) {
    mlp::GemmArgs g{};
    g.A = w.H[l];
    g.lda = L.k[l];
    g.Bt = shadow + L.sw[l];
    g.ldb = L.k[l];
    g.M = B;
    g.N = mlp::WID;
    g.K = L.k[l];
    g.bias = params + L.b[l];
    g.Z = with_train ? w.Z[l] : nullptr;   // pre-activations: only the backward pass reads them
    g.ldz = mlp::WID;
    g.H = w.H[l + 1];
    g.ldh = mlp::WID;
    g.HT = with_train ? w.HT[l + 1] : nullptr;
    g.ldht = B;
    if ((e = gemm<mlp::EPI_FWD>(g, st)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace
}  // namespace drt

using namespace drt;

namespace {
drt_status mlp_fail(drt_status st, const char* msg) {
  set_error_message(msg);
  return st;
}
bool a16(const void* p) { return p && (reinterpret_cast<uintptr_t>(p) & 15) == 0; }
}  // namespace

extern "C" {

drt_status drt_mlp_sizes(int32_t batch, int64_t* n_params, size_t* shadow_bytes,
                         size_t* workspace_bytes) {
  const mlp::Layout L = mlp::layout();
  if (n_params) *n_params = L.total;
  if (shadow_bytes) *shadow_bytes = (size_t)L.stotal * sizeof(mlp::bf16);
  if (workspace_bytes) {
    if (batch < 64 || batch % 64) return mlp_fail(DRT_ERR_INVALID_ARG, "batch must be a positive multiple of 64");
    *workspace_bytes = carve(nullptr, batch).bytes;
  }
  return DRT_OK;
}

drt_status drt_mlp_shadow(const float* params, void* shadow, void* stream) {
  if (!params || !a16(shadow)) return mlp_fail(DRT_ERR_INVALID_ARG, "params / shadow (16-byte aligned)");
  mlp::shadow_kernel<<<256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      params, static_cast<mlp::bf16*>(shadow));
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DRT_OK : mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
}

drt_status drt_mlp_forward(const float* params, const void* shadow, const float* freqs,
                           const float* x, int32_t batch, float* y, void* workspace,
                           size_t workspace_bytes, void* stream) {
  if (!params || !a16(shadow) || !freqs || !x || !y)
    return mlp_fail(DRT_ERR_INVALID_ARG, "NULL or misaligned pointer");
  if (batch < 64 || batch % 64) return mlp_fail(DRT_ERR_INVALID_ARG, "batch must be a positive multiple of 64");
  const MlpWs w = carve(workspace, batch);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < w.bytes)
    return mlp_fail(DRT_ERR_WORKSPACE, "MLP workspace too small or not 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mlp::Layout L = mlp::layout();
  const mlp::bf16* sh = static_cast<const mlp::bf16*>(shadow);
  int* status = g_tc_mode.load() != 0 ? tc_status_ptr() : nullptr;
  if (status) {
    // tcgen05 path: the whole network in one kernel, activations on chip
    mlp::FusedArgs fa{};
    fa.params = params;
    fa.shadow = sh;
    fa.freqs = freqs;
    fa.x = x;
    fa.y = y;
    fa.batch = batch;
    for (int l = 0; l < mlp::NL; ++l) {
      fa.swc[l] = L.swc[l];
      fa.b[l] = L.b[l];
    }
    fa.sw5 = L.sw5;
    fa.b5 = L.b5;
    const int grid = (batch + mlp::FZ_ROWS - 1) / mlp::FZ_ROWS;
    mlp::tc_mlp_forward_kernel<<<grid, mlp::FZ_THREADS, mlp::FZ_SMEM, st>>>(fa, status,
                                                                        g_tc_skip_mma.load());
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DRT_OK : mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaError_t e = mlp_hidden_forward(params, sh, freqs, x, batch, w, false, st);
  if (e == cudaSuccess) {
    mlp::out_layer_kernel<<<std::min(4096, (batch * 32 + 255) / 256), 256, 0, st>>>(
        w.H[mlp::NL], sh + L.sw5, params, L.b5, batch, nullptr, y, nullptr);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? DRT_OK : mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
}

drt_status drt_mlp_loss_grad(const float* params, const void* shadow, const float* freqs,
                             const float* x, const float* target, int32_t batch, float* loss,
                             float* grad, void* workspace, size_t workspace_bytes, void* stream) {
  if (!params || !a16(shadow) || !freqs || !x || !target || !loss || !grad)
    return mlp_fail(DRT_ERR_INVALID_ARG, "NULL or misaligned pointer");
  if (batch < 64 || batch % 64) return mlp_fail(DRT_ERR_INVALID_ARG, "batch must be a positive multiple of 64");
  const MlpWs w = carve(workspace, batch);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < w.bytes)
    return mlp_fail(DRT_ERR_WORKSPACE, "MLP workspace too small or not 256-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const mlp::Layout L = mlp::layout();
  const mlp::bf16* sh = static_cast<const mlp::bf16*>(shadow);
  const int B = batch;
  cudaError_t e = mlp_hidden_forward(params, sh, freqs, x, B, w, true, st);
  if (e != cudaSuccess) return mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
  const int rb = std::min(4096, (B * 32 + 255) / 256);
  mlp::out_layer_kernel<<<rb, 256, 0, st>>>(w.H[mlp::NL], sh + L.sw5, params, L.b5, B, target, w.y, w.dy);
  mlp::loss_reduce_kernel<<<1, 1024, 0, st>>>(w.y, target, w.dy, B, loss, grad + L.b5);
  // d loss / d w5 = sum_b dy[b] h4[b]  (rows of h4^T)
  mlp::row_sum_kernel<<<(mlp::WID * 32 + 255) / 256, 256, 0, st>>>(w.HT[mlp::NL], mlp::WID, B, w.dy,
                                                                   grad + L.w5);
  mlp::out_backward_kernel<<<std::min(4096, (B * mlp::WID + 255) / 256), 256, 0, st>>>(
      w.dy, sh + L.sw5, w.Z[mlp::NL - 1], B, w.dZa, w.dZTa);
  e = cudaGetLastError();
  bf16* dZ = w.dZa;
  bf16* dZT = w.dZTa;
  bf16* dZn = w.dZb;
  bf16* dZTn = w.dZTb;
  for (int l = mlp::NL - 1; l >= 0 && e == cudaSuccess; --l) {
    mlp::GemmArgs g{};
    g.A = dZT;             // [256][B]
    g.lda = B;
    g.Bt = w.HT[l];        // [K_l][B]
    g.ldb = B;
    g.M = mlp::WID;
    g.N = L.k[l];
    g.K = B;
    g.C = w.part;
    g.ldc = L.k[l];
    g.k_splits = w.splits;
    if ((e = gemm<mlp::EPI_DW>(g, st)) != cudaSuccess) break;
    {
      const long long n = (long long)mlp::WID * L.k[l];
      mlp::splitk_reduce_kernel<<<(int)std::min<long long>((n + 255) / 256, 1024), 256, 0, st>>>(
          w.part, w.splits, n, grad + L.w[l]);
      if ((e = cudaGetLastError()) != cudaSuccess) break;
    }
    mlp::row_sum_kernel<<<(mlp::WID * 32 + 255) / 256, 256, 0, st>>>(dZT, mlp::WID, B, nullptr,
                                                                     grad + L.b[l]);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if (l > 0) {
      mlp::GemmArgs h{};
      h.A = dZ;            // [B][256]
      h.lda = mlp::WID;
      h.Bt = sh + L.swt[l];   // W_l^T: [K_l][256]
      h.ldb = mlp::WID;
      h.M = B;
      h.N = L.k[l];
      h.K = mlp::WID;
      h.Z = w.Z[l - 1];
      h.ldz = mlp::WID;
      h.H = dZn;
      h.ldh = mlp::WID;
      h.HT = dZTn;
      h.ldht = B;
      if ((e = gemm<mlp::EPI_DH>(h, st)) != cudaSuccess) break;
      std::swap(dZ, dZn);
      std::swap(dZT, dZTn);
    }
  }
  return e == cudaSuccess ? DRT_OK : mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
}

drt_status drt_mlp_set_tensor_core_path(int32_t use_tcgen05) {
  if (use_tcgen05 < 0 || use_tcgen05 > 2) return mlp_fail(DRT_ERR_INVALID_ARG, "use_tcgen05 must be 0, 1 or 2");
  g_tc_mode.store(use_tcgen05);
  return DRT_OK;
}

drt_status drt_mlp_test_skip_mma(int32_t skip) {
  g_tc_skip_mma.store(skip ? 1 : 0);
  return DRT_OK;
}

drt_status drt_mlp_tc_status(int32_t* timed_out) {
  if (!timed_out) return mlp_fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, mlp::g_tc_status, sizeof(int));
  if (e == cudaSuccess) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(mlp::g_tc_status, &zero, sizeof(int));
  }
  if (e != cudaSuccess) return mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
  *timed_out = v;
  return v ? DRT_ERR_TIMEOUT : DRT_OK;
}

drt_status drt_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t* step,
                        float lr, float beta1, float beta2, float eps, void* shadow, void* stream) {
  if (!params || !m || !v || !grad || !step) return mlp_fail(DRT_ERR_INVALID_ARG, "NULL pointer");
  if (shadow && !a16(shadow)) return mlp_fail(DRT_ERR_INVALID_ARG, "shadow must be 16-byte aligned");
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
    return mlp_fail(DRT_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  mlp::adam_kernel<<<256, 256, 0, st>>>(params, m, v, grad, step, lr, beta1, beta2, eps,
                                        static_cast<mlp::bf16*>(shadow));
  mlp::increment_kernel<<<1, 32, 0, st>>>(step);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DRT_OK : mlp_fail(DRT_ERR_CUDA, cudaGetErrorString(e));
}

}  // extern "C"
