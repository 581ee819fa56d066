// Learned initial guess for the mixture temperature solve (no counterpart in the
// paper; a requirement of the learned form): an 8 -> 64 -> 64 -> 1 tanh MLP that
// maps (normalised e, Y_1..Y_7) to a normalised temperature.
//
//   * training, FP32: per-sample forward and backward passes, gradients summed
//     over each block's samples in shared memory and added to the batch gradient,
//     then an Adam update; samples come from the Newton solver;
//   * inference, FP16 operands with FP32 accumulation on the fifth-generation tensor
//     cores: a block takes 128 nodes as the M = 128 rows of two tcgen05 MMAs (features
//     x W1^T, then tanh(.) x W2^T, accumulators in tensor memory), the activations
//     through the hardware tanh on FP16 pairs; the guess seeds the FP64 Newton solve
//     of the same nodes in the same kernel (dg_newton.cuh), which stays the arbiter and
//     the fallback, to the same |dT| < tol.
//
// Flat parameter layout (float): W1 [64][8] | b1 [64] | W2 [64][64] | b2 [64] | W3 [64] | b3.
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_newton.cuh"
#include "dg_umma.cuh"

namespace dg {
namespace {

constexpr int NI = 8, NH = 64;
constexpr int P_W1 = 0, P_B1 = 512, P_W2 = 576, P_B2 = 4672, P_W3 = 4736, P_B3 = 4800;
static_assert(P_B3 + 1 == DG_MLP_PARAMS, "parameter layout");

// ---- training ----------------------------------------------------------------------------------
constexpr int TS = 128;  // samples per block
constexpr int HS = 65;   // padded row of the per-sample activation tables

__global__ void __launch_bounds__(TS) mlp_grad_kernel(const float* __restrict__ theta, const float* __restrict__ X,
                                                      const float* __restrict__ tgt, int64_t n, float inv_batch,
                                                      float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* sW = sm;                    // DG_MLP_PARAMS
  float* sX = sW + DG_MLP_PARAMS;    // TS x 8
  float* sH1 = sX + TS * NI;         // TS x HS
  float* sH2 = sH1 + TS * HS;
  float* sD1 = sH2 + TS * HS;
  float* sD2 = sD1 + TS * HS;
  float* sdy = sD2 + TS * HS;        // TS
  float* sred = sdy + TS;            // 32
  const int s = threadIdx.x;
  for (int i = s; i < DG_MLP_PARAMS; i += blockDim.x) sW[i] = theta[i];
  const int64_t idx = (int64_t)blockIdx.x * TS + s;
  const bool valid = idx < n;
#pragma unroll
  for (int k = 0; k < NI; ++k) sX[s * NI + k] = valid ? X[idx * NI + k] : 0.0f;
  __syncthreads();
  const float* W1 = sW + P_W1;
  const float* b1 = sW + P_B1;
  const float* W2 = sW + P_W2;
  const float* b2 = sW + P_B2;
  const float* W3 = sW + P_W3;
  float x[NI];
#pragma unroll
  for (int k = 0; k < NI; ++k) x[k] = sX[s * NI + k];
  float h1[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) {
    float a = b1[j];
#pragma unroll
    for (int k = 0; k < NI; ++k) a = fmaf(W1[j * NI + k], x[k], a);
    h1[j] = tanhf(a);
    sH1[s * HS + j] = h1[j];
  }
  float y = sW[P_B3];
  for (int i = 0; i < NH; ++i) {
    float a = b2[i];
#pragma unroll
    for (int j = 0; j < NH; ++j) a = fmaf(W2[i * NH + j], h1[j], a);
    const float h = tanhf(a);
    sH2[s * HS + i] = h;
    y = fmaf(W3[i], h, y);
  }
  const float r = valid ? y - tgt[idx] : 0.0f;
  const float dy = 2.0f * r * inv_batch;
  sdy[s] = dy;
  float d1[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) d1[j] = 0.0f;
  for (int i = 0; i < NH; ++i) {
    const float h = sH2[s * HS + i];
    const float d2 = dy * W3[i] * (1.0f - h * h);
    sD2[s * HS + i] = d2;
#pragma unroll
    for (int j = 0; j < NH; ++j) d1[j] = fmaf(W2[i * NH + j], d2, d1[j]);
  }
#pragma unroll
  for (int j = 0; j < NH; ++j) sD1[s * HS + j] = d1[j] * (1.0f - h1[j] * h1[j]);
  // batch loss
  float l = r * r * inv_batch;
#pragma unroll
  for (int o = 16; o; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((s & 31) == 0) sred[s >> 5] = l;
  __syncthreads();
  if (s == 0) {
    float t = 0.0f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sred[w];
    atomicAdd(loss, t);
  }
  // gradient sums over the block's samples
  for (int e = s; e < DG_MLP_PARAMS; e += blockDim.x) {
    float acc = 0.0f;
    if (e < P_B1) {
      const int j = e / NI, k = e - j * NI;
      for (int t = 0; t < TS; ++t) acc = fmaf(sD1[t * HS + j], sX[t * NI + k], acc);
    } else if (e < P_W2) {
      const int j = e - P_B1;
      for (int t = 0; t < TS; ++t) acc += sD1[t * HS + j];
    } else if (e < P_B2) {
      const int i = (e - P_W2) / NH, j = (e - P_W2) - i * NH;
      for (int t = 0; t < TS; ++t) acc = fmaf(sD2[t * HS + i], sH1[t * HS + j], acc);
    } else if (e < P_W3) {
      const int i = e - P_B2;
      for (int t = 0; t < TS; ++t) acc += sD2[t * HS + i];
    } else if (e < P_B3) {
      const int i = e - P_W3;
      for (int t = 0; t < TS; ++t) acc = fmaf(sdy[t], sH2[t * HS + i], acc);
    } else {
      for (int t = 0; t < TS; ++t) acc += sdy[t];
    }
    atomicAdd(&grad[e], acc);
  }
}

constexpr size_t kGradSmem = sizeof(float) * (DG_MLP_PARAMS + TS * NI + 4 * TS * HS + TS + 32);

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ grad, float* __restrict__ m,
                            float* __restrict__ v, float lr, float bc1, float bc2) {
  // beta1 = 0.9, beta2 = 0.999 and 1 - beta each rounded to FP32 once (1.0f - 0.999f would be
  // 1.3e-5 away from 0.001, and the bias corrections bc1, bc2 are formed from the exact decimals)
  const float b1 = 0.9f, b2 = 0.999f, c1 = 0.1f, c2 = 0.001f, eps = 1e-8f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < DG_MLP_PARAMS; i += gridDim.x * blockDim.x) {
    const float g = grad[i];
    const float mi = fmaf(b1, m[i], c1 * g);
    const float vi = fmaf(b2, v[i], c2 * g * g);
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    grad[i] = 0.0f;
  }
}

// features x = ((e - e_mean)/e_scale, Y_1..Y_ns, 0...), target (T - T_mean)/T_scale
__global__ void features_kernel(int64_t n, int ns, const double* __restrict__ e, const double* __restrict__ Y,
                                const double* __restrict__ T, dg_mlp_norm nrm, float* __restrict__ X,
                                float* __restrict__ t) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    X[i * NI] = (float)((e[i] - nrm.e_mean) / nrm.e_scale);
    for (int k = 0; k < NI - 1; ++k) X[i * NI + 1 + k] = k < ns ? (float)Y[k * n + i] : 0.0f;
    if (T) t[i] = (float)((T[i] - nrm.T_mean) / nrm.T_scale);
  }
}

// ---- inference on the tensor cores, fused with Newton ------------------------------------------
// Operands in shared memory in the UMMA K-major layout without swizzle: 8-row x 16-byte core
// matrices, LBO = 128 B between core matrices adjacent in K, SBO between 8-row groups.
//   A1 [128 nodes][16]: the 8 features (columns 8..15 zero)          SBO 256
//   B1 [64 units][16]:  W1 (input columns 8..15 zero)                  SBO 256
//   A2 [128 nodes][64]: tanh(h1) in FP16                               SBO 1024
//   B2 [64 units][64]:  W2                                             SBO 1024
// MMA 1: D[128][64] = A1 . B1^T (K = 16); MMA 2: D = A2 . B2^T (four K = 16 steps), both into
// the same 64 TMEM columns (the first accumulator is read out before the second MMA is issued).
constexpr int kMlpRows = 128;
constexpr int A1_SBO = 256, A2_SBO = 1024, LBO = 128;
constexpr int W1_IMG = NH / 8 * A1_SBO, W2_IMG = NH / 8 * A2_SBO;  // bytes: 2 KB, 8 KB

__host__ __device__ constexpr int umma_off(int row, int k, int sbo) {
  return (row >> 3) * sbo + (k >> 3) * LBO + (row & 7) * 16 + (k & 7) * 2;
}

// The FP16 weight images (W1 padded to 16 inputs), exactly as the inference block holds them.
__global__ void mlp_image_kernel(const float* __restrict__ theta, __half* __restrict__ w1img,
                                 __half* __restrict__ w2img) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < NH * 16 + NH * NH; i += gridDim.x * blockDim.x) {
    if (i < NH * 16) {
      const int j = i / 16, k = i - j * 16;
      w1img[umma_off(j, k, A1_SBO) / 2] = __float2half_rn(k < NI ? theta[P_W1 + j * NI + k] : 0.0f);
    } else {
      const int i2 = i - NH * 16, r = i2 / NH, k = i2 - r * NH;
      w2img[umma_off(r, k, A2_SBO) / 2] = __float2half_rn(theta[P_W2 + r * NH + k]);
    }
  }
}

// tanh of two floats through the hardware approximation on an FP16 pair (about 11 correct bits:
// the guess only seeds Newton); the result's low half is tanh(lo).
__device__ __forceinline__ uint32_t tanh_pair(float lo, float hi) {
  uint32_t x, y;
  asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(x) : "f"(hi), "f"(lo));
  asm("tanh.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}

__device__ __forceinline__ uint32_t pack_half2(float lo, float hi) {
  return (uint32_t)__half_as_ushort(__float2half_rn(lo)) | ((uint32_t)__half_as_ushort(__float2half_rn(hi)) << 16);
}

struct MlpDev {
  const uint4* w1img;  // [W1_IMG / 16]
  const uint4* w2img;  // [W2_IMG / 16]
  const float* theta;  // fp32 master (biases, W3)
  dg_mlp_norm nrm;
};

// The activations' operands and the Newton state are live at different times of a tile (the MMAs
// have completed before the Newton rounds begin, and the rounds' results are read before the next
// tile's features are written), so they share storage: 31 KB per block, seven blocks per SM.
struct __align__(128) MlpSmem {
  unsigned char B1[W1_IMG];
  unsigned char B2[W2_IMG];
  union {
    struct {
      unsigned char A1[kMlpRows / 8 * A1_SBO];
      unsigned char A2[kMlpRows / 8 * A2_SBO];
    } op;
    newton::Rounds<kMlpRows> R;
  } u;
  float b1[NH], b2[NH], w3[NH];
  uint64_t bar;
  uint32_t tmem;
};
static_assert(sizeof(MlpSmem) <= 32 * 1024, "seven blocks per SM");
constexpr int kMlpBlocksPerSm = 7;

// 128 nodes per tile, one per thread (thread i = MMA row i = TMEM lane i): the node's state and
// species fold (FP2FOLD: the mixed form's float-pair fold), the features, the two MMAs, tanh on
// FP16 pairs, W3 . h2 + b3, the clamped guess, then (unless guess_only) the block's Newton rounds
// from the guesses and the node's outputs.  Fusing the inference with the solve reads the state
// once, and while one block waits for its MMAs the other blocks on the SM keep the FP64 pipe
// busy.  A wait that runs out of polls sets DG_STATUS_TIMEOUT; the block stops at its next issue
// point (decided by a block-wide OR, so every thread stops at the same one), waits once more with
// the full bound for the MMA group that thread 0 issued last, and frees its tensor memory; the
// tiles not reached are not written.
template <bool FP2FOLD>
__global__ void __launch_bounds__(kMlpRows, kMlpBlocksPerSm) temperature_mlp_kernel(
    const GasParams g, const int64_t n, const double* __restrict__ q, double* __restrict__ T,
    int32_t* __restrict__ iters, const MlpDev mlp, const int guess_only, unsigned* __restrict__ status,
    const MixturePrims mp, const int wait_polls) {
  __shared__ MlpSmem S;
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < W1_IMG / 16; i += kMlpRows) reinterpret_cast<uint4*>(S.B1)[i] = mlp.w1img[i];
  for (int i = tid; i < W2_IMG / 16; i += kMlpRows) reinterpret_cast<uint4*>(S.B2)[i] = mlp.w2img[i];
  for (int i = tid; i < NH; i += kMlpRows) {
    S.b1[i] = mlp.theta[P_B1 + i];
    S.b2[i] = mlp.theta[P_B2 + i];
    S.w3[i] = mlp.theta[P_W3 + i];
  }
  const float b3 = mlp.theta[P_B3];
  const float e_mean = (float)mlp.nrm.e_mean, inv_e_scale = (float)(1.0 / mlp.nrm.e_scale);
  if (tid == 0) tc::mbar_init(tc::smem_u32(&S.bar), 1);
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&S.tmem), NH);
  tc::fence_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tm_lane = S.tmem + ((uint32_t)(warp * 32) << 16);  // this warp's quarter of the lanes
  const uint32_t bar = tc::smem_u32(&S.bar);
  constexpr uint32_t IDESC = tc::idesc_f16(kMlpRows, NH);
  uint32_t phase = 0;
  bool timed_out = false;  // this thread saw a wait run out
  bool pending = false;    // thread 0: an issued MMA group it has not yet seen complete
  auto wait = [&]() {
    if (tc::mbar_wait(bar, phase, wait_polls)) {
      if (tid == 0) pending = false;
    } else if (!timed_out) {
      timed_out = true;
      atomicOr(status, (unsigned)DG_STATUS_TIMEOUT);
    }
    phase ^= 1u;
    tc::tc_fence_after();
  };
  const int64_t ntiles = (n + kMlpRows - 1) / kMlpRows;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t i = tile * kMlpRows + tid;
    const bool valid = i < n;
    double rho = 1.0, ir = 1.0, rho_e = 0.0, C[6] = {0, 0, 0, 0, 0, 0}, rhoR = 0.0;
    float feat[NI] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (valid) {
      double rhoY[DG_MAX_SPECIES];
      newton::load_node<FP2FOLD>(g, q, n, i, rho, ir, rho_e, C, rhoR, rhoY);
      feat[0] = (cvt::narrow(rho_e * ir) - e_mean) * inv_e_scale;
      const float irf = cvt::narrow(ir);
#pragma unroll
      for (int k = 0; k < NI - 1; ++k) feat[1 + k] = k < g.ns ? cvt::narrow(rhoY[k]) * irf : 0.0f;
    }
    __syncthreads();  // the previous tile's Newton state (same storage as the operands) has been read
    unsigned char* A1 = S.u.op.A1;
    *reinterpret_cast<uint4*>(A1 + umma_off(tid, 0, A1_SBO)) =
        make_uint4(pack_half2(feat[0], feat[1]), pack_half2(feat[2], feat[3]), pack_half2(feat[4], feat[5]),
                   pack_half2(feat[6], feat[7]));
    *reinterpret_cast<uint4*>(A1 + umma_off(tid, 8, A1_SBO)) = make_uint4(0u, 0u, 0u, 0u);  // K padding
    // layer 1
    tc::fence_async_smem();
    tc::tc_fence_before();
    if (__syncthreads_or(timed_out)) break;
    if (tid == 0) {
      tc::tc_fence_after();
      tc::mma_f16(S.tmem, tc::umma_desc(tc::smem_u32(A1), LBO, A1_SBO), tc::umma_desc(tc::smem_u32(S.B1), LBO,
                                                                                      A1_SBO),
                  IDESC, 0u);
      tc::mma_commit(bar);
      pending = true;
    }
    wait();
    {
      float acc[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        tc::tmem_ld32(tm_lane + (uint32_t)(32 * half), acc);
        uint32_t w[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          w[j] = tanh_pair(acc[2 * j] + S.b1[32 * half + 2 * j], acc[2 * j + 1] + S.b1[32 * half + 2 * j + 1]);
#pragma unroll
        for (int c = 0; c < 4; ++c)
          *reinterpret_cast<uint4*>(S.u.op.A2 + umma_off(tid, 32 * half + 8 * c, A2_SBO)) =
              make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
      }
    }
    // layer 2
    tc::fence_async_smem();
    tc::tc_fence_before();
    if (__syncthreads_or(timed_out)) break;
    if (tid == 0) {
      tc::tc_fence_after();
#pragma unroll
      for (int ks = 0; ks < NH / 16; ++ks)
        tc::mma_f16(S.tmem, tc::umma_desc(tc::smem_u32(S.u.op.A2) + ks * 2 * LBO, LBO, A2_SBO),
                    tc::umma_desc(tc::smem_u32(S.B2) + ks * 2 * LBO, LBO, A2_SBO), IDESC, ks > 0 ? 1u : 0u);
      tc::mma_commit(bar);
      pending = true;
    }
    wait();
    float y = b3;
    {
      float acc[32];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        tc::tmem_ld32(tm_lane + (uint32_t)(32 * half), acc);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int u = 32 * half + 2 * j;
          const uint32_t h = tanh_pair(acc[2 * j] + S.b2[u], acc[2 * j + 1] + S.b2[u + 1]);
          const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&h));
          y = fmaf(S.w3[u], hf.x, fmaf(S.w3[u + 1], hf.y, y));
        }
      }
    }
    double t = fma(mlp.nrm.T_scale, (double)y, mlp.nrm.T_mean);
    t = fmin(fmax(t, mlp.nrm.T_min), mlp.nrm.T_max);
    if (guess_only) {
      if (valid) T[i] = t;
      continue;
    }
    newton::stage(S.u.R, valid, C, rho_e, t);
    if (newton::rounds(S.u.R, g.newton_max_it, g.newton_tol) && tid == 0)
      atomicOr(status, DG_STATUS_NO_CONVERGENCE);
    if (!valid) continue;
    t = S.u.R.t[tid];
    T[i] = t;
    if (iters) iters[i] = S.u.R.it[tid];
    if (mp.rec || mp.prim) {
      const double rhocv = newton::heat_capacity(C, t);
      if (mp.rec) newton::store_prims(mp, g, q, n, i, rho, ir, rhoR, t, rhocv);
      if (mp.prim) newton::store_prims64(mp, n, i, rho, ir, rhoR, t, rhocv);
    }
  }
  // an MMA group whose wait ran out for thread 0 (parity phase ^ 1: phase flipped after the wait)
  // may still be in flight: one more wait, with the full bound, before the accumulator is released
  if (tid == 0 && pending) tc::mbar_wait(bar, phase ^ 1u);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(S.tmem, NH);
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

cudaError_t ensure_half_weights(dg_gas gas) {
  if (!gas->mlp_w1h) {
    cudaError_t e = cudaMalloc((void**)&gas->mlp_w1h, W1_IMG);
    if (e == cudaSuccess) e = cudaMalloc((void**)&gas->mlp_w2h, W2_IMG);
    if (e != cudaSuccess) return e;
  }
  mlp_image_kernel<<<16, 256>>>(gas->mlp_theta, (__half*)gas->mlp_w1h, (__half*)gas->mlp_w2h);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e;
}

}  // namespace

cudaError_t launch_temperature_mlp(dg_gas gas, int64_t n, const double* q, double* T, int32_t* iters, int guess_only,
                                   cudaStream_t s, const MixturePrims& mp, int wait_polls) {
  if (n <= 0) return cudaSuccess;
  MlpDev m{(const uint4*)gas->mlp_w1h, (const uint4*)gas->mlp_w2h, gas->mlp_theta, gas->mlp_norm};
  // the mixed-precision form (node records out) folds the species in float pairs
  const bool fp2 = mp.rec != nullptr;
  static int per_sm[2] = {0, 0};
  if (!per_sm[fp2])
    per_sm[fp2] = std::max(1, resident_blocks(fp2 ? (const void*)temperature_mlp_kernel<true>
                                                  : (const void*)temperature_mlp_kernel<false>, kMlpRows, 0, NH));
  const int64_t tiles = (n + kMlpRows - 1) / kMlpRows;
  const int blocks = (int)std::min<int64_t>(tiles, (int64_t)per_sm[fp2] * device_sms());
  const int polls = wait_polls > 0 ? wait_polls : tc::kWaitPolls;
  if (fp2)
    temperature_mlp_kernel<true><<<blocks, kMlpRows, 0, s>>>(gas->p, n, q, T, iters, m, guess_only, gas->status, mp,
                                                             polls);
  else
    temperature_mlp_kernel<false><<<blocks, kMlpRows, 0, s>>>(gas->p, n, q, T, iters, m, guess_only, gas->status,
                                                              mp, polls);
  return cudaGetLastError();
}

cudaError_t mlp_set_params(dg_gas gas, const float* theta_host, const dg_mlp_norm& nrm) {
  cudaError_t e = cudaSuccess;
  if (!gas->mlp_theta) e = cudaMalloc((void**)&gas->mlp_theta, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess)
    e = cudaMemcpy(gas->mlp_theta, theta_host, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = ensure_half_weights(gas);
  if (e == cudaSuccess) {
    gas->mlp_norm = nrm;
    gas->has_mlp = true;
  }
  return e;
}

cudaError_t mlp_loss_grad(int64_t n, const float* theta, const float* X, const float* t, float* grad, float* loss,
                          cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGradSmem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t blocks = (n + TS - 1) / TS;
  mlp_grad_kernel<<<(unsigned)blocks, TS, kGradSmem, s>>>(theta, X, t, n, 1.0f / (float)n, grad, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam_step(int t, float lr, float* theta, float* grad, float* m, float* v, cudaStream_t s) {
  // bias corrections 1 - beta^t formed in FP64 and rounded once
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)t)), bc2 = (float)(1.0 - std::pow(0.999, (double)t));
  adam_kernel<<<(DG_MLP_PARAMS + 255) / 256, 256, 0, s>>>(theta, grad, m, v, lr, bc1, bc2);
  return cudaGetLastError();
}

cudaError_t mlp_train(dg_gas gas, int64_t n, const double* e_dev, const double* Y_dev, const double* T_dev,
                      const dg_mlp_train_opts& o, const float* init_host, float* history) {
  // normalisation from the data (host copies of e and T)
  std::vector<double> he(n), hT(n);
  cudaError_t e = cudaMemcpy(he.data(), e_dev, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(hT.data(), T_dev, sizeof(double) * n, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  dg_mlp_norm nrm;
  std::memset(&nrm, 0, sizeof(nrm));
  double se = 0, se2 = 0, sT = 0, sT2 = 0, Tmin = hT[0], Tmax = hT[0];
  for (int64_t i = 0; i < n; ++i) {
    se += he[i];
    se2 += he[i] * he[i];
    sT += hT[i];
    sT2 += hT[i] * hT[i];
    Tmin = std::min(Tmin, hT[i]);
    Tmax = std::max(Tmax, hT[i]);
  }
  nrm.e_mean = se / n;
  nrm.e_scale = std::sqrt(std::max(se2 / n - nrm.e_mean * nrm.e_mean, 1e-300));
  nrm.T_mean = sT / n;
  nrm.T_scale = std::sqrt(std::max(sT2 / n - nrm.T_mean * nrm.T_mean, 1e-300));
  nrm.T_min = Tmin;
  nrm.T_max = Tmax;
  float *X = nullptr, *t = nullptr, *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr, *loss = nullptr;
  e = cudaMalloc((void**)&X, sizeof(float) * NI * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&t, sizeof(float) * n);
  if (e == cudaSuccess) e = cudaMalloc((void**)&theta, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&grad, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&m, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&v, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMalloc((void**)&loss, sizeof(float));
  if (e == cudaSuccess) e = cudaMemcpy(theta, init_host, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(grad, 0, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMemset(m, 0, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) e = cudaMemset(v, 0, sizeof(float) * DG_MLP_PARAMS);
  if (e == cudaSuccess) {
    features_kernel<<<sm_count() * 8, 256>>>(n, gas->p.ns, e_dev, Y_dev, T_dev, nrm, X, t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)kGradSmem);
  const int64_t batch = o.batch;
  const int64_t nb = n / batch;  // full batches only
  int64_t step = 0;
  float lr = o.lr;
  for (int ep = 0; ep < o.epochs && e == cudaSuccess; ++ep) {
    e = cudaMemset(loss, 0, sizeof(float));
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
      const int64_t off = ((b + (int64_t)ep * 7919) % nb) * batch;  // batch order rotates per epoch
      mlp_grad_kernel<<<(unsigned)((batch + TS - 1) / TS), TS, kGradSmem>>>(theta, X + off * NI, t + off, batch,
                                                                             1.0f / (float)batch, grad, loss);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = mlp_adam_step((int)std::min<int64_t>(++step, 1 << 30), lr, theta, grad, m, v, 0);
    }
    float l = 0.0f;
    if (e == cudaSuccess) e = cudaMemcpy(&l, loss, sizeof(float), cudaMemcpyDeviceToHost);
    if (history) history[ep] = l / (float)std::max<int64_t>(nb, 1);
    lr *= o.lr_decay;
  }
  std::vector<float> trained(DG_MLP_PARAMS);
  if (e == cudaSuccess)
    e = cudaMemcpy(trained.data(), theta, sizeof(float) * DG_MLP_PARAMS, cudaMemcpyDeviceToHost);
  cudaFree(X);
  cudaFree(t);
  cudaFree(theta);
  cudaFree(grad);
  cudaFree(m);
  cudaFree(v);
  cudaFree(loss);
  if (e == cudaSuccess) e = mlp_set_params(gas, trained.data(), nrm);
  return e;
}

}  // namespace dg
