// Cardinality model: a 3-layer MLP (32 -> 128 -> 128 -> 1, ReLU) that predicts the log growth
// of the intermediate table for a candidate join step, trained on the cardinalities the
// executor logs. Matmuls run on the tensor cores as BF16 x BF16 -> FP32 (tcgen05.mma with the
// accumulator in tensor memory); the
// master weights, biases, the output layer and Adam's moments stay FP32. Activations that
// feed a matmul are rounded to BF16 (round to nearest even) right after they are produced.
//
// Flat parameter layout (FP32): W1[128][32] | b1[128] | W2[128][128] | b2[128] | w3[128] | b3.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "kernels.h"

namespace dmk {

constexpr int MLP_IN = 32, MLP_H = 128;

// C[M x N] (+)= sum_k A(m, k) * B(k, n); A(m, k) = A[m * am + k * ak], B(k, n) = B[k * bk + n * bn],
// M % 16 == 0, N = 32 or 128, K % 16 == 0: fifth-generation tensor cores (tcgen05). A CTA of 16
// warps owns 128 rows of C; its accumulator is 128 lanes x N FP32 columns of tensor memory. Per
// K chunk of up to 256 (a training batch of 256 samples is one chunk) the CTA stages A (its 128
// rows, zero past M) and B (N rows, as B^T) in shared memory in the canonical K-major layout
// without swizzle -- 8 x 8 BF16 core matrices of 128 contiguous bytes, 128 bytes apart along K
// and 4 KB apart along M / N -- and one thread issues the chunk's K / 16 MMAs (M = 128, K = 16
// each) and commits them to an mbarrier that every thread waits on before the next chunk is
// staged. Warp w then reads 32 columns (group w / 4) of the accumulator lanes 32 (w % 4) ..
// 32 (w % 4) + 31 (tcgen05.ld) and writes them to its rows of C. Every wait is bounded: a chunk
// whose MMAs do not complete within about a second raises *err, and the CTA still waits (bounded
// again) for them before it frees its tensor memory.
constexpr int TC_M = 128, TC_KC = 256, TC_THREADS = 512, TC_COLS = 128;
// shared memory of a CTA: A and B chunks (64 KB each; a whole training batch of 256 samples is
// one chunk). At 512 threads at most 4 CTAs could share an SM (2048 threads), so their tensor
// memory (4 x 128 of 512 columns) is always free to allocate.
constexpr int TC_SMEM = 2 * TC_M * TC_KC * 2;
static_assert(2048 / TC_THREADS * TC_COLS <= 512, "resident CTAs could exhaust tensor memory");
constexpr long long TC_WAIT_CYCLES = 2000000000ll;

__device__ __forceinline__ uint32_t tc_saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// BF16 offset of element (r, k) of a staged operand: core matrix (r / 8, k / 8), then row-major
// inside it.
__device__ __forceinline__ int tc_core_off(int r, int k) {
  return (((r >> 3) * (TC_KC >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M / N) byte offsets
// between core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, N, M = 128.
__device__ __forceinline__ uint32_t tc_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);
}

// Spins with the non-blocking test (the MMAs of a chunk take microseconds; a suspending wait
// could sleep past their completion).
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > TC_WAIT_CYCLES) return false;
  }
}

__global__ void __launch_bounds__(TC_THREADS) k_gemm_tc(int M, int N, int K, const __nv_bfloat16 *A, int am, int ak,
                                                        const __nv_bfloat16 *Bm, int bk, int bn, float *C, int ldc,
                                                        int accumulate, unsigned *err) {
  extern __shared__ __align__(1024) uint16_t tc_smem[];
  uint16_t *sA = tc_smem, *sB = tc_smem + TC_M * TC_KC;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M;
  const int kb = 0, ke = K;
  const uint32_t bar_a = tc_saddr(&bar);
  if (warp == 0) {  // the accumulator: 128 lanes x TC_COLS columns
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_saddr(&tmem_base)),
                 "r"(TC_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = tc_idesc(N);
  const bool vecA = ak == 1 && am % 8 == 0 && ((uintptr_t)A & 15) == 0;
  const bool vecB = bk == 1 && bn % 8 == 0 && ((uintptr_t)Bm & 15) == 0;
  const bool tA = am == 1 && ak % 8 == 0 && ((uintptr_t)A & 15) == 0;
  const bool tB = bn == 1 && bk % 8 == 0 && ((uintptr_t)Bm & 15) == 0;
  const uint32_t sbo = (TC_KC >> 3) * 128;  // bytes between 8-row groups
  uint32_t phase = 0;
  bool ok = true;
  for (int k0 = kb; k0 < ke && ok; k0 += TC_KC) {
    const int kc = min(TC_KC, ke - k0);  // a multiple of 16
    // an operand whose K is contiguous (16-byte aligned rows) moves as 16-byte pieces, one core
    // matrix row each; otherwise consecutive threads take consecutive elements of its contiguous
    // dimension
    // thread order: the 8 rows of a core matrix are 8 neighbouring threads (128 contiguous
    // bytes of shared memory: no bank conflict), then the core matrices along K, then along M
    if (vecA) {
      for (int i = tid; i < TC_M * (kc >> 3); i += TC_THREADS) {
        const int rest = i >> 3, kp = rest % (kc >> 3);
        const int r = ((rest / (kc >> 3)) << 3) | (i & 7), k = kp << 3;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (m0 + r < M) v = *(const uint4 *)(A + (int64_t)(m0 + r) * am + k0 + k);
        *(uint4 *)(sA + tc_core_off(r, k)) = v;
      }
    } else if (tA) {  // M contiguous: 16-byte pieces of 8 rows at one k, scattered to the rows
      for (int i = tid; i < kc * (TC_M >> 3); i += TC_THREADS) {  // neighbouring threads: neighbouring k
        const int r = (i / kc) << 3, k = i % kc;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (m0 + r < M) v = *(const uint4 *)(A + m0 + r + (int64_t)(k0 + k) * ak);  // M % 8 == 0
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 8; j++) sA[tc_core_off(r + j, k)] = (uint16_t)(w[j >> 1] >> (16 * (j & 1)));
      }
    } else {
      for (int i = tid; i < TC_M * kc; i += TC_THREADS) {
        const int r = am == 1 ? i % TC_M : i / kc, k = am == 1 ? i / TC_M : i % kc;
        sA[tc_core_off(r, k)] =
            m0 + r < M ? __bfloat16_as_ushort(A[(int64_t)(m0 + r) * am + (int64_t)(k0 + k) * ak]) : (uint16_t)0;
      }
    }
    if (vecB) {
      for (int i = tid; i < N * (kc >> 3); i += TC_THREADS) {
        const int rest = i >> 3, kp = rest % (kc >> 3);
        const int n = ((rest / (kc >> 3)) << 3) | (i & 7), k = kp << 3;
        *(uint4 *)(sB + tc_core_off(n, k)) = *(const uint4 *)(Bm + (int64_t)n * bn + k0 + k);
      }
    } else if (tB) {  // N contiguous: 16-byte pieces of 8 columns at one k
      for (int i = tid; i < kc * (N >> 3); i += TC_THREADS) {
        const int n = (i / kc) << 3, k = i % kc;
        const uint4 v = *(const uint4 *)(Bm + (int64_t)(k0 + k) * bk + n);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 8; j++) sB[tc_core_off(n + j, k)] = (uint16_t)(w[j >> 1] >> (16 * (j & 1)));
      }
    } else {
      for (int i = tid; i < N * kc; i += TC_THREADS) {
        const int n = bn == 1 ? i % N : i / kc, k = bn == 1 ? i / N : i % kc;
        sB[tc_core_off(n, k)] = __bfloat16_as_ushort(Bm[(int64_t)(k0 + k) * bk + (int64_t)n * bn]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tensor cores read what was stored
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      for (int kk = 0; kk < kc; kk += 16) {
        const uint64_t ad = tc_sdesc(tc_saddr(sA) + (kk >> 3) * 128, 128, sbo);
        const uint64_t bd = tc_sdesc(tc_saddr(sB) + (kk >> 3) * 128, 128, sbo);
        const uint32_t acc = (k0 + kk) > kb;  // the CTA's first MMA overwrites the accumulator
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                   : "memory");
    }
    const bool landed = tc_wait(bar_a, phase);  // the chunk's MMAs are done with sA and sB
    phase ^= 1u;
    ok = __syncthreads_and(landed);
    if (!ok) {
      if (tid == 0) atomicOr(err, 1u);
      tc_wait(bar_a, phase ^ 1u);  // let them finish (bounded) before the memory is freed
    }
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int quad = warp & 3, c0 = 32 * (warp >> 2);  // a warp reads its lane quadrant (warp % 4)
  if (ok && kb < ke && c0 < N) {  // rows m0 + 32 quad + lane, columns c0 .. c0 + 31
    const int row = m0 + 32 * quad + lane;
    {
      uint32_t v[32];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
          "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < M) {  // the row's 32 columns as 16-byte pieces (ldc % 4 == 0, C 16-byte aligned)
        float4 *c = (float4 *)(C + (int64_t)row * ldc + c0);
#pragma unroll
        for (int j = 0; j < 8; j++) {
          float4 x = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                 __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
          if (accumulate) {
            const float4 o = c[j];
            x.x += o.x;
            x.y += o.y;
            x.z += o.z;
            x.w += o.w;
          }
          c[j] = x;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS) : "memory");
  if (tid == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar_a) : "memory");
}

__global__ void k_to_bf16(const float *x, __nv_bfloat16 *y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16_rn(x[i]);
}

// H = relu(Z + b) rounded to BF16; Z keeps the pre-activation (its sign is the ReLU mask).
__global__ void k_bias_relu(float *Z, const float *b, __nv_bfloat16 *H, int rows, int cols) {
  int64_t n = (int64_t)rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float z = Z[i] + b[i % cols];
    Z[i] = z;
    H[i] = __float2bfloat16_rn(z > 0.f ? z : 0.f);
  }
}

// y[r] = sum_o H2[r][o] * w3[o] + b3 (FP32); with targets, dy[r] = 2 (y - t) / n_valid for valid rows
// and the squared error is added to *loss.
__global__ void k_out_layer(const __nv_bfloat16 *H2, const float *w3, const float *b3, int rows, int n_valid,
                            const float *target, float *y, float *dy, float *loss) {
  int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (r >= rows) return;
  float s = 0.f;
  for (int o = lane; o < MLP_H; o += 32) s += __bfloat162float(H2[(int64_t)r * MLP_H + o]) * w3[o];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if (lane == 0) {
    float v = s + b3[0];
    y[r] = v;
    if (target) {
      float e = r < n_valid ? v - target[r] : 0.f;
      dy[r] = 2.f * e / (float)n_valid;
      if (r < n_valid) atomicAdd(loss, e * e / (float)n_valid);
    }
  }
}

// Column sums of a rows x cols matrix, 32 columns a block: warp w of 8 adds rows w, w + 8, ...
// of its lane's column (coalesced), and the 8 partial sums are added in a fixed order.
template <typename T>
__device__ __forceinline__ float colsum32(const T *M, const float *wrow, int rows, int cols, int c,
                                          float *s_part) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  float s = 0.f;
  if (c < cols)
    for (int r = w; r < rows; r += 8) {
      float x;
      if constexpr (sizeof(T) == 2) x = __bfloat162float(M[(int64_t)r * cols + c]);
      else x = (float)M[(int64_t)r * cols + c];
      s += wrow ? wrow[r] * x : x;
    }
  s_part[w * 32 + l] = s;
  __syncthreads();
  float t = 0.f;
  if (w == 0)
    for (int k = 0; k < 8; k++) t += s_part[k * 32 + l];
  __syncthreads();
  return t;  // valid in warp 0
}

// dH2 = dy * w3 masked by Z2 > 0 (BF16), every block over its grid-stride share; blocks 0 .. 3
// also add dw3 (32 columns each) and block 0 db3 (FP32, accumulated). 256 threads a block.
__global__ void k_out_backward(const float *dy, const __nv_bfloat16 *H2, const float *Z2, const float *w3, int rows,
                               __nv_bfloat16 *dH2, float *dw3, float *db3) {
  __shared__ float s_part[256];
  if (blockIdx.x < MLP_H / 32) {
    const int c = blockIdx.x * 32 + (threadIdx.x & 31);
    const float t = colsum32(H2, dy, rows, MLP_H, c, s_part);
    if (threadIdx.x < 32) dw3[c] += t;
    if (blockIdx.x == 0) {
      const float u = colsum32(dy, (const float *)nullptr, rows, 1, threadIdx.x & 31, s_part);
      if (threadIdx.x == 0) db3[0] += u;
    }
  }
  int64_t n = (int64_t)rows * MLP_H;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i / MLP_H;
    int oo = (int)(i - r * MLP_H);
    float g = Z2[i] > 0.f ? dy[r] * w3[oo] : 0.f;
    dH2[i] = __float2bfloat16_rn(g);
  }
}

// dH = dA masked by Z > 0, rounded to BF16.
__global__ void k_relu_backward(const float *dA, const float *Z, __nv_bfloat16 *dH, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dH[i] = __float2bfloat16_rn(Z[i] > 0.f ? dA[i] : 0.f);
}

// db[c] += sum_r dH[r][c]: 32 columns a block of 256 threads
__global__ void k_colsum(const __nv_bfloat16 *dH, int rows, int cols, float *db) {
  __shared__ float s_part[256];
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const float t = colsum32(dH, (const float *)nullptr, rows, cols, c, s_part);
  if (threadIdx.x < 32 && c < cols) db[c] += t;
}

__global__ void k_adam(float *w, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

static int blocks_for(int64_t n, int per = 256) {
  int64_t b = (n + per - 1) / per;
  return (int)(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

static cudaError_t gemm(int M, int N, int K, const __nv_bfloat16 *A, int am, int ak, const __nv_bfloat16 *Bm, int bk,
                        int bn, float *C, int ldc, int acc, unsigned *err, cudaStream_t s) {
  if (M % 16 || K % 16 || (N != 32 && N != 128) || ldc % 4 || ((uintptr_t)C & 15)) return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> attr_set{0};  // one bit per device ordinal below 64
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (!bit || !(attr_set.load() & bit)) {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    attr_set.fetch_or(bit);
  }
  g_launches++;
  k_gemm_tc<<<(M + TC_M - 1) / TC_M, TC_THREADS, TC_SMEM, s>>>(M, N, K, A, am, ak, Bm, bk, bn, C, ldc, acc, err);
  return cudaGetLastError();
}

int64_t mlp_param_count() { return (int64_t)MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1; }

int64_t mlp_work_bytes(int rows) {
  int64_t r = rows;
  return r * MLP_IN * 2 + 2 * (r * MLP_H * 4) + 2 * (r * MLP_H * 2) + 3 * r * 4 + 2 * (r * MLP_H * 2) +
         r * MLP_H * 4 + 2 * mlp_param_count() * 2 + 4096 + 256;
}

unsigned *mlp_error_flag(void *work, int rows) {
  return (unsigned *)((unsigned char *)work + (mlp_work_bytes(rows) - 256) / 256 * 256);
}

// Forward (and, with targets, backward into grads) for `rows` samples (rows % 16 == 0; the
// first n_valid are real). X: rows x 32 FP32 on the device; params / grads: flat FP32.
cudaError_t mlp_forward_backward(const float *params, const float *X, const float *target, int rows, int n_valid,
                                 float *y, float *grads, float *loss, void *work, cudaStream_t s) {
  const float *W1 = params, *b1 = W1 + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H;
  const float *w3 = b2 + MLP_H, *b3 = w3 + MLP_H;
  unsigned char *p = (unsigned char *)work;
  auto take = [&](int64_t bytes) {
    void *q = p;
    p += (bytes + 255) / 256 * 256;
    return q;
  };
  __nv_bfloat16 *Xb = (__nv_bfloat16 *)take((int64_t)rows * MLP_IN * 2);
  float *Z1 = (float *)take((int64_t)rows * MLP_H * 4);
  float *Z2 = (float *)take((int64_t)rows * MLP_H * 4);
  __nv_bfloat16 *H1 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  __nv_bfloat16 *H2 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  float *dy = (float *)take((int64_t)rows * 4);
  __nv_bfloat16 *dH2 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  __nv_bfloat16 *dH1 = (__nv_bfloat16 *)take((int64_t)rows * MLP_H * 2);
  float *dA1 = (float *)take((int64_t)rows * MLP_H * 4);
  __nv_bfloat16 *W1b = (__nv_bfloat16 *)take((int64_t)MLP_H * MLP_IN * 2);
  __nv_bfloat16 *W2b = (__nv_bfloat16 *)take((int64_t)MLP_H * MLP_H * 2);
  unsigned *err = mlp_error_flag(work, rows);  // raised by a tensor-core wait that ran out
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int launches = 0;
  k_to_bf16<<<blocks_for((int64_t)rows * MLP_IN), 256, 0, s>>>(X, Xb, (int64_t)rows * MLP_IN);
  k_to_bf16<<<blocks_for(MLP_H * MLP_IN), 256, 0, s>>>(W1, W1b, MLP_H * MLP_IN);
  k_to_bf16<<<blocks_for(MLP_H * MLP_H), 256, 0, s>>>(W2, W2b, MLP_H * MLP_H);
  launches += 3;
  // Z1 = X W1^T: A = X (row-major), B(k, n) = W1[n][k]
  e = gemm(rows, MLP_H, MLP_IN, Xb, MLP_IN, 1, W1b, 1, MLP_IN, Z1, MLP_H, 0, err, s);
  if (e != cudaSuccess) return e;
  k_bias_relu<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(Z1, b1, H1, rows, MLP_H);
  e = gemm(rows, MLP_H, MLP_H, H1, MLP_H, 1, W2b, 1, MLP_H, Z2, MLP_H, 0, err, s);
  if (e != cudaSuccess) return e;
  k_bias_relu<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(Z2, b2, H2, rows, MLP_H);
  k_out_layer<<<(rows + 7) / 8, 256, 0, s>>>(H2, w3, b3, rows, n_valid, target, y, dy, loss);
  launches += 3;
  if (target && grads) {
    float *gW1 = grads, *gb1 = gW1 + MLP_H * MLP_IN, *gW2 = gb1 + MLP_H, *gb2 = gW2 + MLP_H * MLP_H;
    float *gw3 = gb2 + MLP_H, *gb3 = gw3 + MLP_H;
    k_out_backward<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(dy, H2, Z2, w3, rows, dH2, gw3, gb3);
    k_colsum<<<MLP_H / 32, 256, 0, s>>>(dH2, rows, MLP_H, gb2);
    launches += 2;
    // gW2[o][i] += sum_r dH2[r][o] H1[r][i]: A(m=o, k=r) = dH2[r][o], B(k=r, n=i) = H1[r][i]
    e = gemm(MLP_H, MLP_H, rows, dH2, 1, MLP_H, H1, MLP_H, 1, gW2, MLP_H, 1, err, s);
    if (e != cudaSuccess) return e;
    // dA1[r][i] = sum_o dH2[r][o] W2[o][i]: A = dH2 (row-major), B(k=o, n=i) = W2[o][i]
    e = gemm(rows, MLP_H, MLP_H, dH2, MLP_H, 1, W2b, MLP_H, 1, dA1, MLP_H, 0, err, s);
    if (e != cudaSuccess) return e;
    k_relu_backward<<<blocks_for((int64_t)rows * MLP_H), 256, 0, s>>>(dA1, Z1, dH1, (int64_t)rows * MLP_H);
    k_colsum<<<MLP_H / 32, 256, 0, s>>>(dH1, rows, MLP_H, gb1);
    launches += 2;
    // gW1[o][j] += sum_r dH1[r][o] X[r][j]
    e = gemm(MLP_H, MLP_IN, rows, dH1, 1, MLP_H, Xb, MLP_IN, 1, gW1, MLP_IN, 1, err, s);
    if (e != cudaSuccess) return e;
  }
  g_launches += launches;
  return cudaGetLastError();
}

cudaError_t mlp_adam(float *params, const float *grads, float *m, float *v, int64_t n, float lr, int step,
                     cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f;
  float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  g_launches++;
  k_adam<<<blocks_for(n), 256, 0, s>>>(params, grads, m, v, n, lr, b1, b2, 1e-8f, c1, c2);
  return cudaGetLastError();
}

}  // namespace dmk
