// Neural-field MLP on the 5th-generation tensor cores (tcgen05), 16-bit operands (FP16 or
// BF16), FP32 accumulation in tensor memory (arXiv 2509.03623, Methods, "Neural Temperature Recovery":
// T(r,|z|) = MLP_w(gamma(r,|z|)) with a sinusoidal encoding gamma; the network shape here is
// 64 Fourier features -> 4 x 128 SiLU -> 4 outputs).
//
// One persistent CTA per SM (two tile groups of 8 warps, ~185 KB of shared memory); the
// groups work on different tiles so that one group's MMAs overlap the other's epilogue. At
// start the CTA converts the FP32 master weights to 16 bits into shared memory in the
// no-swizzle K-major "core matrix" layout (8 rows x 16 bytes per core matrix) and allocates
// 128 columns of tensor memory per group. Per tile of 128 samples, with two warps on each
// TMEM lane quadrant (one per half of the columns, so row m belongs to two threads):
//   the two threads of row m compute half of the features of sample m each (range-reduced
//   sin/cos) into the A buffer;
//   one thread issues the K/16 tcgen05.mma of the layer (M=128, N=128 or 16 for the last
//   layer) and commits them to an mbarrier; every thread waits (bounded), reads its half of
//   the accumulator row back with tcgen05.ld, adds the bias, applies SiLU in packed 16-bit
//   arithmetic and writes the activations in place into the A buffer for the next layer;
//   after the last layer one thread per row writes the 4 FP32 outputs.
// Ray setups (double precision) come from a pre-pass, one thread per ray.
// Waits on the mbarrier are bounded: on expiry the CTA records an error and stops after
// releasing its tensor memory.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "rt_internal.cuh"

namespace rtb {

constexpr int kMlpF = 64;      // features (2 x 32 Fourier directions)
constexpr int kMlpW = 128;     // hidden width
constexpr int kMlpOut = 4;     // outputs
constexpr int kMlpOutPad = 16; // last layer padded to the smallest MMA N
constexpr int kMlpTile = 128;  // samples per tile (MMA M)
constexpr unsigned kSpinLimit = 1u << 26;

struct MlpParamsDev {
  const float *B;     // [32][2]
  const float *W[5];  // [out][in] fp32
  const float *b[5];
};

// 16-bit operands (BF16 or FP16 bit patterns, chosen by the kernel's F16 parameter).
typedef unsigned short h16;

constexpr int kTG = 2;        // tile groups per CTA, one tile in flight per group
constexpr int kGW = 8;        // warps per group: two per TMEM lane quadrant (column halves)
constexpr int kGT = kGW * 32; // threads per group

struct __align__(1024) MlpSmem {
  h16 W1[kMlpW * kMlpF];          // 16 KB
  h16 Wh[3][kMlpW * kMlpW];       // 96 KB
  h16 W5[kMlpOutPad * kMlpW];     // 4 KB
  h16 A[kTG][kMlpTile * kMlpW];   // 2 x 32 KB, one activation buffer per tile group
  float bias[4][kMlpW];
  float bias5[kMlpOutPad];
  float Bf[32][2];
  unsigned long long mbar[kTG];
  unsigned tmem_base;
  int abort[kTG];  // per tile group: written before, read after the group's barrier
};

static __device__ int g_mlp_error;  // set when a bounded wait expires

// Element offset of (row r, column k) in a rows x K tile stored as core matrices of 8 rows x 8
// bf16 (16 bytes), core matrix (r/8, k/8) at ((r/8) (K/8) + k/8) x 64 elements.
__device__ __forceinline__ int cm_off(int r, int k, int K) {
  return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7);
}

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// tcgen05 shared-memory matrix descriptor, no swizzle, K-major: LBO = distance between core
// matrices along K (128 B), SBO = distance between 8-row groups ((K/8) x 128 B).
__device__ __forceinline__ unsigned long long mma_desc(unsigned addr, int K) {
  unsigned long long lbo = 128 >> 4, sbo = (unsigned long long)((K >> 3) * 128) >> 4;
  return (unsigned long long)((addr >> 4) & 0x3FFF) | ((lbo & 0x3FFF) << 16) |
         ((sbo & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16 (format 1) or FP16 (format 0),
// both K-major, M = 128.
__host__ __device__ constexpr unsigned idesc_16(int N, bool f16) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((unsigned)(N >> 3) << 17) | ((128u >> 4) << 24);
}

template <bool F16>
__device__ __forceinline__ h16 to16(float x) {
  if (F16) return __half_as_ushort(__float2half_rn(x));
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

__device__ __forceinline__ void mma_bf16(unsigned tmem_d, unsigned long long a,
                                         unsigned long long b, unsigned idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(unsigned mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait(unsigned mbar, unsigned phase) {
  for (unsigned it = 0; it < kSpinLimit; it++) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float *v) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float *v) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

// SiLU(x) = x sigma(x) = 0.5 x (1 + tanh(x/2)) (hardware tanh; the result is rounded to BF16).
__device__ __forceinline__ float silu(float x) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * x));
  float h = 0.5f * x;
  return fmaf(h, t, h);
}

// SiLU of two pre-activations in the 16-bit format, packed: h = z/2 (exact), t = tanh(h)
// (hardware, packed), SiLU = h + h t (one packed FMA); the result is the next layer's operand.
template <bool F16>
__device__ __forceinline__ unsigned silu2(float z0, float z1) {
  unsigned z, h, t, r;
  if (F16) {
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(z) : "f"(z1), "f"(z0));
    asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(h) : "r"(z), "r"(0x38003800u));
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(h), "r"(t), "r"(h));
  } else {
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(z) : "f"(z1), "f"(z0));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(h) : "r"(z), "r"(0x3F003F00u));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(h), "r"(t), "r"(h));
  }
  return r;
}

// Store 8 consecutive 16-bit values of row m starting at column k (k multiple of 8).
template <bool F16>
__device__ __forceinline__ void store8(h16 *A, int m, int k, int K, const float *v) {
  unsigned p[4];
#pragma unroll
  for (int j = 0; j < 4; j++)
    p[j] = (unsigned)to16<F16>(v[2 * j]) | ((unsigned)to16<F16>(v[2 * j + 1]) << 16);
  *reinterpret_cast<uint4 *>(A + cm_off(m, k, K)) = make_uint4(p[0], p[1], p[2], p[3]);
}

// Fourier features of x = (rhat, zhat) for directions [16 half, 16 half + 16):
// sin 2 pi B x into f[0..15], cos into f[16..31]; phases reduced to [-1/2, 1/2) cycles before
// the hardware sin/cos.
__device__ __forceinline__ void features(const MlpSmem &S, float rh, float zh, int half,
                                         float *f) {
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const int i = 16 * half + j;
    float ph = fmaf(S.Bf[i][0], rh, S.Bf[i][1] * zh);
    ph -= rintf(ph);
    float a = 6.283185307179586f * ph;
    f[j] = __sinf(a);
    f[16 + j] = __cosf(a);
  }
}

// Input suppliers: the network inputs of sample s0 + tid of a tile (false when the sample
// needs no evaluation). Called by every thread of the CTA.
struct XYInput {
  const float *xy;
  long long n;
};

__device__ __forceinline__ bool tile_input(const XYInput &in, Ray *, long long s0, int tid,
                                           float *rh, float *zh, int) {
  long long s = s0 + tid;
  if (s >= in.n) return false;
  float2 v = reinterpret_cast<const float2 *>(in.xy)[s];
  *rh = v.x;
  *zh = v.y;
  return true;
}

// Samples of rays: s = pixel * n_samples + k; the ray setups come from a pre-pass (one thread
// per ray, double precision) in device memory.
struct RayInput {
  MarchParams P;
  const Ray *rays;
};

__device__ __forceinline__ void sample_coords(const MarchParams &P, const Ray &R, int k,
                                              bool *gas, float *rh, float *zh) {
  float kf = (float)k;
  float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  Cell c = locate(P, z, fmaf(R.x, R.x, y * y));
  *gas = c.gas && R.hit;
  *rh = ((float)c.i0 + c.fr) / (float)(P.nr - 1);
  *zh = c.zr / P.zr_max;
}

__device__ __forceinline__ bool tile_input(const RayInput &in, Ray *, long long s0, int tid,
                                           float *rh, float *zh, int) {
  const MarchParams &P = in.P;
  const long long n = (long long)P.nx * P.ny * P.n_samples;
  long long s = s0 + tid;
  if (s >= n) return false;
  const Ray R = in.rays[s / P.n_samples];
  bool gas;
  sample_coords(P, R, (int)(s % P.n_samples), &gas, rh, zh);
  return gas;
}

// Ray setups of every pixel (one thread per ray).
__global__ void rays_kernel(const __grid_constant__ MarchParams P, Ray *__restrict__ rays) {
  const long long npix = (long long)P.nx * P.ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix < npix) rays[pix] = setup_ray(P, (int)(pix % P.nx), (int)(pix / P.nx), true);
}

template <class In, bool F16>
__global__ void __launch_bounds__(kGT * kTG, 1)
    mlp_tc_kernel(const MlpParamsDev Wp, const __grid_constant__ In in, float *__restrict__ out,
                  long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  MlpSmem &S = *reinterpret_cast<MlpSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int tg = tid / kGT;                       // tile group
  const int q = warp & 3;                         // TMEM lane quadrant of this warp
  const int half = (warp >> 2) & 1;               // column half handled by this warp
  const int t = q * 32 + (tid & 31);              // row (= sample) of the tile
  const int gt = tid % kGT;                       // thread index within the group
  Ray *rays = nullptr;

  // ---- one-time setup: weights to the 16-bit core-matrix layout, biases, TMEM, mbarriers ----
  const int nt = blockDim.x;
  for (int i = tid; i < kMlpW * kMlpF; i += nt) {
    int o = i / kMlpF, k = i % kMlpF;
    S.W1[cm_off(o, k, kMlpF)] = to16<F16>(Wp.W[0][i]);
  }
  for (int l = 0; l < 3; l++)
    for (int i = tid; i < kMlpW * kMlpW; i += nt) {
      int o = i / kMlpW, k = i % kMlpW;
      S.Wh[l][cm_off(o, k, kMlpW)] = to16<F16>(Wp.W[l + 1][i]);
    }
  for (int i = tid; i < kMlpOutPad * kMlpW; i += nt) {
    int o = i / kMlpW, k = i % kMlpW;
    S.W5[cm_off(o, k, kMlpW)] = to16<F16>(o < kMlpOut ? Wp.W[4][o * kMlpW + k] : 0.0f);
  }
  for (int i = tid; i < 4 * kMlpW; i += nt) S.bias[i / kMlpW][i % kMlpW] = Wp.b[i / kMlpW][i % kMlpW];
  if (tid < kMlpOutPad) S.bias5[tid] = tid < kMlpOut ? Wp.b[4][tid] : 0.0f;
  if (tid < 64) S.Bf[tid >> 1][tid & 1] = Wp.B[tid];
  if (tid == 0) {
    for (int g = 0; g < kTG; g++) S.abort[g] = 0;
    for (int g = 0; g < kTG; g++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar[g])), "r"(1));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(128 * kTG));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = S.tmem_base + 128 * tg;             // this group's columns
  const unsigned tlane = tmem + ((unsigned)(q * 32) << 16);  // this warp's lanes
  const unsigned mbar = smem_u32(&S.mbar[tg]);
  h16 *A = S.A[tg];
  const unsigned aA = smem_u32(A);
  unsigned phase = 0;
  // named barrier of the tile group (ids 1, 2; 0 is __syncthreads)
  auto gsync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + tg), "r"(kGT) : "memory"); };

  const long long ntiles = (n + kMlpTile - 1) / kMlpTile;
  for (long long tile = (long long)blockIdx.x * kTG + tg; tile < ntiles;
       tile += (long long)gridDim.x * kTG) {
    const long long s = tile * kMlpTile + t;
    float rh = 0.0f, zh = 0.0f;
    const bool need = tile_input(in, rays, tile * kMlpTile, t, &rh, &zh, tg);
    // any sample of the tile needs the network? (group-wide vote through shared memory)
    int any;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(any)
        : "r"((unsigned)need), "r"(1 + tg), "r"(kGT)
        : "memory");
    if (!any) continue;
    {
      float f[32];
      features(S, rh, zh, half, f);
      store8<F16>(A, t, 16 * half, kMlpF, f);
      store8<F16>(A, t, 16 * half + 8, kMlpF, f + 8);
      store8<F16>(A, t, 32 + 16 * half, kMlpF, f + 16);
      store8<F16>(A, t, 32 + 16 * half + 8, kMlpF, f + 24);
    }
    proxy_fence();
    tc_fence_before();
    gsync();
    bool ok = true;
    for (int l = 0; l < 5 && ok; l++) {
      const int K = l == 0 ? kMlpF : kMlpW;
      const int N = l == 4 ? kMlpOutPad : kMlpW;
      if (gt == 0) {
        tc_fence_after();
        const unsigned bB =
            l == 0 ? smem_u32(S.W1) : (l == 4 ? smem_u32(S.W5) : smem_u32(S.Wh[l - 1]));
        for (int ks = 0; ks < K / 16; ks++)
          mma_bf16(tmem, mma_desc(aA + ks * 256, K), mma_desc(bB + ks * 256, K), idesc_16(N, F16),
                   ks > 0);
        mma_commit(mbar);
      }
      ok = mbar_wait(mbar, phase);
      phase ^= 1;
      tc_fence_after();
      if (!ok) {
        S.abort[tg] = 1;
        atomicExch(&g_mlp_error, 1);
      }
      if (ok && l < 4) {
#pragma unroll
        for (int c0 = 64 * half; c0 < 64 * half + 64; c0 += 32) {
          float v[32];
          tmem_ld32(tlane + c0, v);
          unsigned p[16];
#pragma unroll
          for (int j = 0; j < 16; j++)
            p[j] = silu2<F16>(v[2 * j] + S.bias[l][c0 + 2 * j], v[2 * j + 1] + S.bias[l][c0 + 2 * j + 1]);
#pragma unroll
          for (int k = 0; k < 4; k++)
            *reinterpret_cast<uint4 *>(A + cm_off(t, c0 + 8 * k, kMlpW)) =
                make_uint4(p[4 * k], p[4 * k + 1], p[4 * k + 2], p[4 * k + 3]);
        }
      } else if (ok) {
        float v[16];
        tmem_ld16(tlane, v);
        if (need && half == 0) {
          float4 o = make_float4(v[0] + S.bias5[0], v[1] + S.bias5[1], v[2] + S.bias5[2],
                                 v[3] + S.bias5[3]);
          reinterpret_cast<float4 *>(out)[s] = o;
        }
      }
      proxy_fence();
      tc_fence_before();
      gsync();
      ok = !S.abort[tg];
    }
    if (S.abort[tg]) break;
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem_base),
                 "r"(128 * kTG));
  }
}

int mlp_validate(const rt_mlp *m);
static int mlp_check(const rt_mlp *m) { return mlp_validate(m); }

int mlp_validate(const rt_mlp *m) {
  if (!m) return set_error(RT_EINVAL, "null network");
  if (m->n_freq != 32 || m->width != kMlpW || m->hidden != 4 || m->n_out != kMlpOut)
    return set_error(RT_EINVAL, "network shape must be 32 Fourier directions, 4 hidden layers "
                     "of 128, 4 outputs (got %d, %d x %d, %d)", m->n_freq, m->hidden, m->width,
                     m->n_out);
  if (!m->B) return set_error(RT_EINVAL, "null Fourier directions");
  if (m->precision != RT_MLP_F16 && m->precision != RT_MLP_BF16)
    return set_error(RT_EINVAL, "precision must be RT_MLP_F16 or RT_MLP_BF16");
  for (int l = 0; l < 5; l++)
    if (!m->W[l] || !m->b[l]) return set_error(RT_EINVAL, "null weight or bias of layer %d", l);
  return RT_OK;
}

static MlpParamsDev mlp_dev(const rt_mlp *m) {
  MlpParamsDev d;
  d.B = m->B;
  for (int l = 0; l < 5; l++) {
    d.W[l] = m->W[l];
    d.b[l] = m->b[l];
  }
  return d;
}

template <class In, bool F16>
static int launch_mlp_t(const rt_mlp *m, const In &in, float *out, long long n,
                        cudaStream_t stream) {
  auto kern = mlp_tc_kernel<In, F16>;
  size_t smem = sizeof(MlpSmem);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "mlp smem attribute: %s", cudaGetErrorString(e));
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  long long tiles = (n + kMlpTile - 1) / kMlpTile;
  long long groups = (tiles + kTG - 1) / kTG;
  long long blocks = groups < nsm ? groups : nsm;
  kern<<<(unsigned)blocks, kGT * kTG, smem, stream>>>(mlp_dev(m), in, out, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "mlp launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

template <class In>
static int launch_mlp(const rt_mlp *m, const In &in, float *out, long long n,
                      cudaStream_t stream) {
  if (n <= 0) return RT_OK;
  return m->precision == RT_MLP_BF16 ? launch_mlp_t<In, false>(m, in, out, n, stream)
                                     : launch_mlp_t<In, true>(m, in, out, n, stream);
}

int launch_mlp_rays(const rt_mlp *m, const MarchParams &P, float4 *mod, void *ray_buf,
                    cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  long long n = npix * P.n_samples;
  if (n == 0) return RT_OK;
  Ray *rays = reinterpret_cast<Ray *>(ray_buf);
  rays_kernel<<<(unsigned)((npix + 127) / 128), 128, 0, stream>>>(P, rays);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "ray setup launch: %s", cudaGetErrorString(e));
  RayInput in;
  in.P = P;
  in.rays = rays;
  return launch_mlp(m, in, reinterpret_cast<float *>(mod), n, stream);
}

size_t ray_buffer_bytes(long long npix) { return (size_t)npix * sizeof(Ray); }

// Network inputs (rhat, zhat) of every (pixel, sample): [npix][n_samples] float2, (-1, -1)
// where the sample has no gas.
__global__ void coords_kernel(const __grid_constant__ MarchParams P, float2 *__restrict__ xy) {
  const long long npix = (long long)P.nx * P.ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  Ray R = setup_ray(P, (int)(pix % P.nx), (int)(pix / P.nx), true);
  for (int k = 0; k < P.n_samples; k++) {
    bool gas;
    float rh, zh;
    sample_coords(P, R, k, &gas, &rh, &zh);
    xy[pix * P.n_samples + k] = gas ? make_float2(rh, zh) : make_float2(-1.0f, -1.0f);
  }
}

int launch_coords(const MarchParams &P, float2 *xy, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0) return RT_OK;
  coords_kernel<<<(unsigned)((npix + 127) / 128), 128, 0, stream>>>(P, xy);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "coords launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rtb

using namespace rtb;

extern "C" int rt_mlp_eval(const rt_mlp *mlp, const float *xy, float *out, long long n,
                           void *stream) {
  int rc = mlp_check(mlp);
  if (rc == RT_OK && n < 0) rc = set_error(RT_EINVAL, "negative sample count");
  if (rc == RT_OK && n > 0 && (!xy || !out)) rc = set_error(RT_EINVAL, "null input or output");
  if (rc == RT_OK) rc = launch_mlp(mlp, XYInput{xy, n}, out, n, (cudaStream_t)stream);
  if (rc == RT_OK) clear_error();
  return rc;
}

extern "C" int rt_mlp_status(int *timed_out) {
  if (!timed_out) return set_error(RT_EINVAL, "null output");
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_mlp_error, sizeof(int));
  if (e != cudaSuccess) return set_error(RT_ECUDA, "mlp status: %s", cudaGetErrorString(e));
  *timed_out = v;
  return RT_OK;
}
