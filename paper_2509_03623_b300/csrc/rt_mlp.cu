// Neural-field MLP on the 5th-generation tensor cores (tcgen05), 16-bit operands (FP16 or
// BF16), FP32 accumulation in tensor memory (arXiv 2509.03623, Methods, "Neural Temperature Recovery":
// T(r,|z|) = MLP_w(gamma(r,|z|)) with a sinusoidal encoding gamma; the network shape here is
// 64 Fourier features -> 4 x 128 SiLU -> 4 outputs).
//
// One persistent CTA per SM (three tile groups of 8 warps, ~215 KB of shared memory); the
// groups work on different tiles so that one group's MMAs overlap the others' epilogues. At
// start the CTA converts the FP32 master weights to 16 bits into shared memory in the
// no-swizzle K-major "core matrix" layout (8 rows x 16 bytes per core matrix) and allocates
// tensor memory, 128 columns per group. Per tile of 128 samples, with two warps on each
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

constexpr int kTG = 3;        // tile groups per CTA, one tile in flight per group
constexpr int kGW = 8;        // warps per group: two per TMEM lane quadrant (column halves)
constexpr int kGT = kGW * 32; // threads per group
// tensor-memory columns allocated (a power of two holding 128 per group)
constexpr int kTmemCols = kTG <= 2 ? 256 : 512;

struct __align__(1024) MlpSmem {
  h16 W1[kMlpW * kMlpF];          // 16 KB
  h16 Wh[3][kMlpW * kMlpW];       // 96 KB
  h16 W5[kMlpOutPad * kMlpW];     // 4 KB
  h16 A[kTG][kMlpTile * kMlpW];   // 32 KB per tile group
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
// M = 128; A (bit 15) and B (bit 16) K-major (0) or MN-major (1).
__host__ __device__ constexpr unsigned idesc_16(int N, bool f16, bool a_mn = false,
                                                bool b_mn = false) {
  return (1u << 4) | ((f16 ? 0u : 1u) << 7) | ((f16 ? 0u : 1u) << 10) |
         ((a_mn ? 1u : 0u) << 15) | ((b_mn ? 1u : 0u) << 16) | ((unsigned)(N >> 3) << 17) |
         ((128u >> 4) << 24);
}

// Shared-memory matrix descriptor, no swizzle, MN-major: the 16-byte rows of a core matrix run
// along M (or N), its 8 rows along K; mn_stride and k_stride are the distances between core
// matrices along MN and along K. Without swizzling the leading-dimension offset is the K
// stride and the stride-dimension offset the MN stride, in either major order.
__device__ __forceinline__ unsigned long long mma_desc_mn(unsigned addr, unsigned mn_stride,
                                                          unsigned k_stride) {
  unsigned long long lbo = k_stride >> 4, sbo = mn_stride >> 4;
  return (unsigned long long)((addr >> 4) & 0x3FFF) | ((lbo & 0x3FFF) << 16) |
         ((sbo & 0x3FFF) << 32) | (1ull << 46);
}

// Shared-memory addresses stay below 2^18 bytes, so the 14-bit start-address field of a
// descriptor never wraps: the descriptor of addr + 16 j is the descriptor of addr plus j. The
// MMA issue loops below step descriptors this way (one 64-bit add per instruction), which
// keeps the single issuing thread off a long dependent chain per MMA.
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

// Two FP32 values rounded to the 16-bit format and packed (a in the low half).
template <bool F16>
__device__ __forceinline__ unsigned pack16(float a, float b) {
  unsigned z;
  if (F16)
    asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(z) : "f"(b), "f"(a));
  else
    asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(z) : "f"(b), "f"(a));
  return z;
}

template <bool F16>
__device__ __forceinline__ float2 unpack16(unsigned z) {
  if (F16) {
    __half2 h = *reinterpret_cast<__half2 *>(&z);
    return __half22float2(h);
  }
  __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162 *>(&z);
  return __bfloat1622float2(h);
}

// SiLU of two packed 16-bit pre-activations: h = z/2 (exact), t = tanh(h) (hardware, packed),
// SiLU = h + h t (one packed FMA); the result is the next layer's operand.
template <bool F16>
__device__ __forceinline__ unsigned silu2p(unsigned z) {
  unsigned h, t, r;
  if (F16) {
    asm("mul.rn.f16x2 %0, %1, %2;" : "=r"(h) : "r"(z), "r"(0x38003800u));
    asm("tanh.approx.f16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.f16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(h), "r"(t), "r"(h));
  } else {
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(h) : "r"(z), "r"(0x3F003F00u));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(h));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(r) : "r"(h), "r"(t), "r"(h));
  }
  return r;
}

template <bool F16>
__device__ __forceinline__ unsigned silu2(float z0, float z1) {
  return silu2p<F16>(pack16<F16>(z0, z1));
}

// SiLU'(z) = s (1 + z (1 - s)), s = sigma(z) = (1 + tanh(z/2)) / 2.
__device__ __forceinline__ float dsilu(float z) {
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(0.5f * z));
  const float s = fmaf(0.5f, t, 0.5f);
  return s * fmaf(z, 1.0f - s, 1.0f);
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
__device__ __forceinline__ void features(const float (*Bf)[2], float rh, float zh, int half,
                                         float *f) {
#pragma unroll
  for (int j = 0; j < 16; j++) {
    const int i = 16 * half + j;
    float ph = fmaf(Bf[i][0], rh, Bf[i][1] * zh);
    ph -= rintf(ph);
    float a = 6.283185307179586f * ph;
    f[j] = __sinf(a);
    f[16 + j] = __cosf(a);
  }
}

// Input suppliers: the network inputs of row `tid` of the tile starting at s0 (false when
// the row needs no evaluation) and the index of its output / output gradient. Called by every
// thread of the CTA; in_count bounds the rows.
struct XYInput {
  const float *xy;
  long long n;
};

__device__ __forceinline__ long long in_count(const XYInput &in, long long n) { return n; }

__device__ __forceinline__ bool tile_input(const XYInput &in, long long s0, int tid, float *rh,
                                           float *zh, long long *idx) {
  long long s = s0 + tid;
  *idx = s;
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

__device__ __forceinline__ long long in_count(const RayInput &in, long long n) { return n; }

__device__ __forceinline__ bool tile_input(const RayInput &in, long long s0, int tid, float *rh,
                                           float *zh, long long *idx) {
  const MarchParams &P = in.P;
  const long long n = (long long)P.nx * P.ny * P.n_samples;
  long long s = s0 + tid;
  *idx = s;
  if (s >= n) return false;
  const Ray R = in.rays[s / P.n_samples];
  bool gas;
  sample_coords(P, R, (int)(s % P.n_samples), &gas, rh, zh);
  return gas;
}

// Only the samples with gas, in ray order: list[i] = pixel * n_samples + k (built by
// build_sample_list), *count of them.
struct ListInput {
  MarchParams P;
  const Ray *rays;
  const unsigned *list;
  const unsigned *count;
};

__device__ __forceinline__ long long in_count(const ListInput &in, long long) { return *in.count; }

__device__ __forceinline__ bool tile_input(const ListInput &in, long long s0, int tid, float *rh,
                                           float *zh, long long *idx) {
  const long long s = s0 + tid;
  *idx = 0;
  if (s >= (long long)*in.count) return false;
  const unsigned v = in.list[s];
  const unsigned ns = (unsigned)in.P.n_samples;
  *idx = v;
  bool gas;
  sample_coords(in.P, in.rays[v / ns], (int)(v % ns), &gas, rh, zh);
  return gas;
}

// The listed samples with their inputs and output gradients already gathered in list order
// (gather_list_kernel): xy[i] and g[i], padded with zeros to whole 64-sample tiles, so a row
// needs one load and no bound check.
struct PackedInput {
  const float2 *xy;
  const unsigned *count;
};

__device__ __forceinline__ long long in_count(const PackedInput &in, long long) { return *in.count; }

__device__ __forceinline__ bool tile_input(const PackedInput &in, long long s0, int tid, float *rh,
                                           float *zh, long long *idx) {
  const long long s = s0 + tid;
  *idx = s;
  const float2 v = in.xy[s];
  *rh = v.x;
  *zh = v.y;
  return true;
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
                 "r"(kTmemCols));
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

  const long long ntiles = (in_count(in, n) + kMlpTile - 1) / kMlpTile;
  for (long long tile = (long long)blockIdx.x * kTG + tg; tile < ntiles;
       tile += (long long)gridDim.x * kTG) {
    long long s;
    float rh = 0.0f, zh = 0.0f;
    const bool need = tile_input(in, tile * kMlpTile, t, &rh, &zh, &s);
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
      features(S.Bf, rh, zh, half, f);
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
        const unsigned long long dA = mma_desc(aA, K), dB = mma_desc(bB, K);
        const unsigned id = N == kMlpW ? idesc_16(kMlpW, F16) : idesc_16(kMlpOutPad, F16);
        for (int ks = 0; ks < K / 16; ks++)
          mma_bf16(tmem, dA + 16u * ks, dB + 16u * ks, id, ks > 0);
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
                 "r"(kTmemCols));
  }
}

static_assert(sizeof(MlpSmem) <= 227 * 1024, "shared memory");
static_assert(128 * kTG <= kTmemCols && kTmemCols <= 512, "tensor memory");

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

// ---------------------------------------------------------------------------------------
// BF16 network forward with split operands: the product of every layer is formed as
// W_hi a_hi + W_hi a_lo + W_lo a_hi, where x_hi = bf16(x) and x_lo = x - x_hi for the weights
// W and the activations a (the inputs of each layer, Fourier features included), so the
// rounding of both operands to BF16 (2^-9 relative) drops out to second order. The two
// correction products are about 2^-8 of the main one, so 3 significant bits suffice for
// their factors: they run as FP8 (E5M2, whose 5-bit exponent holds the small low parts
// without scaling) MMAs of K = 32, at twice the BF16 rate, so a K step of 32 costs two BF16
// MMAs and two FP8 MMAs instead of six BF16 MMAs. SiLU is evaluated in FP32 (hardware tanh)
// and the output layer (128 -> 4) runs on the CUDA cores in FP32. The accumulation is FP32 in
// tensor memory throughout.
//
// The product is taken transposed, D[out feature][sample] = W[out][in] a[in][sample], so that
// the weights are the A operand: W_hi of every layer stays in shared memory (BF16, K-major
// core matrices, 112 KB) and E5M2 copies of W and of W_lo in tensor memory (A from tensor
// memory: row o in lane o, four E5M2 per 32-bit column, the lower input in the low byte;
// 224 columns), which leaves shared memory for three tile groups of 64 samples. A group's
// activations are the B operand: a_hi in BF16 (MN-major core matrices of 8 features x 8
// samples, 16 KB) and E5M2 copies of a and of a_lo (MN-major core matrices of 8 features x
// 16 samples, 8 KB each); one thread per (output feature, half of the samples) reads its
// accumulator row back, adds the bias, applies SiLU and writes the next layer's three
// operands in place. After the fourth layer the FP32 activations
// go to shared memory (XOR-swizzled, 32 KB); four threads per sample each form the four
// outputs over a quarter of the 128 inputs in FP32, and one adds the quarters.
// ---------------------------------------------------------------------------------------
constexpr int kSN = 64;                     // samples per tile (MMA N)
constexpr int kSG = 3;                      // tile groups
constexpr int kSGT = 256;                   // threads per group (two per TMEM lane row)
constexpr unsigned kColW8 = 0;              // E5M2 of W: W1 16 columns, W2..W4 32 each
constexpr unsigned kColWlo8 = 112;          // E5M2 of W_lo, the same layout
constexpr unsigned kColSplitD = 224;        // accumulators: 64 columns per group

struct __align__(1024) SplitSmem {
  h16 W1[kMlpW * kMlpF];                 // high parts, K-major core matrices (16 KB)
  h16 Wh[3][kMlpW * kMlpW];              // (96 KB)
  h16 B[kSG][2][kMlpW * kSN];            // activations per group: high, low parts (16 KB each)
  float4 W5T[kMlpW];                     // output layer, transposed: W5T[k] = W5[0..3][k]
  float bias[4][kMlpW];
  float bias5[kMlpOut];
  float Bf[32][2];
  float rh[kSG][kSN], zh[kSG][kSN];
  long long idx[kSG][kSN];
  int need[kSG][kSN];
  unsigned long long mbar[kSG];
  unsigned tmem_base;
  int abort[kSG];
};
static_assert(sizeof(SplitSmem) <= 227 * 1024, "shared memory");
static_assert(kColSplitD + 64 * kSG <= 512, "tensor memory");
static_assert(kColWlo8 + 112 <= kColSplitD, "FP8 weight columns");
// TMEM column of layer l's E5M2 weights (l = 0: W1, 64 inputs; l >= 1: 128 inputs)
__device__ __forceinline__ unsigned col8(unsigned base, int l) {
  return base + (l == 0 ? 0u : 16u + 32u * (unsigned)(l - 1));
}
// the FP32 activations of the last hidden layer fill a group's two activation buffers
static_assert(sizeof(float) * kMlpW * kSN == 2 * sizeof(h16) * kMlpW * kSN, "h4 staging");

// Element offset of (feature k, sample s) in an MN-major B tile: core matrix (k/8, s/8) at
// ((k/8) (kSN/8) + s/8) x 64 elements, row k % 8, element s % 8.
__device__ __forceinline__ int bmn_off(int k, int s) {
  return (((k >> 3) * (kSN >> 3) + (s >> 3)) << 6) + ((k & 7) << 3) + (s & 7);
}

// Byte offset of (feature k, sample s) in an 8-bit MN-major B tile: core matrix (k/8, s/16) of
// 8 features x 16 samples at ((k/8) (kSN/16) + s/16) x 128 bytes, row k % 8, byte s % 16.
__device__ __forceinline__ int b8_off(int k, int s) {
  return (((k >> 3) * (kSN >> 4) + (s >> 4)) << 7) + ((k & 7) << 4) + (s & 15);
}

// four floats to E5M2 (round to nearest, saturating), x0 in the low byte
__device__ __forceinline__ unsigned e5m2x4(float x0, float x1, float x2, float x3) {
  unsigned short lo, hi;
  asm("cvt.rn.satfinite.e5m2x2.f32 %0, %1, %2;" : "=h"(lo) : "f"(x1), "f"(x0));
  asm("cvt.rn.satfinite.e5m2x2.f32 %0, %1, %2;" : "=h"(hi) : "f"(x3), "f"(x2));
  return (unsigned)lo | ((unsigned)hi << 16);
}

// bf16 pair (low half = first) to two floats
__device__ __forceinline__ float2 bf2f(unsigned u) {
  return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
}

// 8 values of feature k at samples s0..s0+7 (s0 multiple of 8): the BF16 high part into Bh and
// E5M2 copies of the value and of its low part into B8 and B8l (8 bytes each)
__device__ __forceinline__ void split_store8(h16 *Bh, unsigned char *B8, unsigned char *B8l,
                                             int k, int s0, const float *v) {
  unsigned hi[4];
  float lo[8];
#pragma unroll
  for (int j = 0; j < 4; j++) {
    hi[j] = pack16<false>(v[2 * j], v[2 * j + 1]);
    const float2 r = __ffma2_rn(bf2f(hi[j]), make_float2(-1.0f, -1.0f),
                                make_float2(v[2 * j], v[2 * j + 1]));  // exact residual
    lo[2 * j] = r.x;
    lo[2 * j + 1] = r.y;
  }
  *reinterpret_cast<uint4 *>(Bh + bmn_off(k, s0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  const int o8 = b8_off(k, s0);
  *reinterpret_cast<uint2 *>(B8 + o8) =
      make_uint2(e5m2x4(v[0], v[1], v[2], v[3]), e5m2x4(v[4], v[5], v[6], v[7]));
  *reinterpret_cast<uint2 *>(B8l + o8) =
      make_uint2(e5m2x4(lo[0], lo[1], lo[2], lo[3]), e5m2x4(lo[4], lo[5], lo[6], lo[7]));
}

// 32 consecutive 32-bit columns of this warp's TMEM lanes from registers
__device__ __forceinline__ void tmem_st32(unsigned taddr, const unsigned *r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// 16 consecutive 32-bit columns of this warp's TMEM lanes from registers
__device__ __forceinline__ void tmem_st16(unsigned taddr, const unsigned *r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}

// 16 values of feature k at samples s0..s0+15 (s0 multiple of 16): the BF16 high part into Bh
// (two rows of 8 samples) and E5M2 copies of the value and of its low part into B8 and B8l
// (one full 16-byte core-matrix row each, so the lanes of a warp store whole rows)
__device__ __forceinline__ void split_store16(h16 *Bh, unsigned char *B8, unsigned char *B8l,
                                              int k, int s0, const float *v) {
  unsigned hi[8];
  float lo[16];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    hi[j] = pack16<false>(v[2 * j], v[2 * j + 1]);
    const float2 r = __ffma2_rn(bf2f(hi[j]), make_float2(-1.0f, -1.0f),
                                make_float2(v[2 * j], v[2 * j + 1]));  // exact residual
    lo[2 * j] = r.x;
    lo[2 * j + 1] = r.y;
  }
  *reinterpret_cast<uint4 *>(Bh + bmn_off(k, s0)) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<uint4 *>(Bh + bmn_off(k, s0 + 8)) = make_uint4(hi[4], hi[5], hi[6], hi[7]);
  const int o8 = b8_off(k, s0);
  *reinterpret_cast<uint4 *>(B8 + o8) =
      make_uint4(e5m2x4(v[0], v[1], v[2], v[3]), e5m2x4(v[4], v[5], v[6], v[7]),
                 e5m2x4(v[8], v[9], v[10], v[11]), e5m2x4(v[12], v[13], v[14], v[15]));
  *reinterpret_cast<uint4 *>(B8l + o8) =
      make_uint4(e5m2x4(lo[0], lo[1], lo[2], lo[3]), e5m2x4(lo[4], lo[5], lo[6], lo[7]),
                 e5m2x4(lo[8], lo[9], lo[10], lo[11]), e5m2x4(lo[12], lo[13], lo[14], lo[15]));
}

// D (tmem) += A (tmem) x B (smem descriptor), 8-bit operands (K = 32); the format fields of the
// instruction descriptor read as E5M2 for this kind
__device__ __forceinline__ void mma_f8_tmem_a(unsigned tmem_d, unsigned tmem_a,
                                              unsigned long long b, unsigned idesc, int accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}\n" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accum));
}

template <class In>
__global__ void __launch_bounds__(kSGT * kSG, 1)
    mlp_split_kernel(const MlpParamsDev Wp, const __grid_constant__ In in,
                     float *__restrict__ out, long long n) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  SplitSmem &S = *reinterpret_cast<SplitSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tg = tid / kSGT;            // tile group
  const int gt = tid % kSGT;            // thread within the group
  const int q = warp & 3;               // TMEM lane quadrant
  const int hs = (warp >> 2) & 1;       // half of the tile's samples
  const int f = q * 32 + lane;          // output feature (TMEM lane) of this thread

  // ---- one-time setup: high parts to shared memory, low parts to tensor memory ----
  for (int i = tid; i < kMlpW * kMlpF; i += blockDim.x)
    S.W1[cm_off(i / kMlpF, i % kMlpF, kMlpF)] = to16<false>(Wp.W[0][i]);
  for (int l = 0; l < 3; l++)
    for (int i = tid; i < kMlpW * kMlpW; i += blockDim.x)
      S.Wh[l][cm_off(i / kMlpW, i % kMlpW, kMlpW)] = to16<false>(Wp.W[l + 1][i]);
  for (int k = tid; k < kMlpW; k += blockDim.x)
    S.W5T[k] = make_float4(Wp.W[4][k], Wp.W[4][kMlpW + k], Wp.W[4][2 * kMlpW + k],
                           Wp.W[4][3 * kMlpW + k]);
  for (int i = tid; i < 4 * kMlpW; i += blockDim.x) S.bias[i / kMlpW][i % kMlpW] = Wp.b[i / kMlpW][i % kMlpW];
  if (tid < kMlpOut) S.bias5[tid] = Wp.b[4][tid];
  if (tid < 64) S.Bf[tid >> 1][tid & 1] = Wp.B[tid];
  if (tid == 0) {
    for (int g = 0; g < kSG; g++) S.abort[g] = 0;
    for (int g = 0; g < kSG; g++)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar[g])), "r"(1));
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = S.tmem_base;
  if (warp < 4) {
    // warp w writes rows 32w..32w+31 (row o = lane o) of the E5M2 copies of W and of W_lo:
    // 16 columns for W1 (64 inputs), 32 for each hidden layer, four inputs per column
    const unsigned trow = tbase + ((unsigned)(warp * 32) << 16);
    const int o = warp * 32 + lane;
    auto lo = [](float a) { return a - __bfloat162float(__float2bfloat16_rn(a)); };
    for (int l = 0; l < 4; l++) {
      const int K = l == 0 ? kMlpF : kMlpW;
      const float *w = Wp.W[l] + (size_t)o * K;
      unsigned rh[32], rl[32];
#pragma unroll
      for (int c = 0; c < 32; c++) {
        if (4 * c < K) {
          rh[c] = e5m2x4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
          rl[c] = e5m2x4(lo(w[4 * c]), lo(w[4 * c + 1]), lo(w[4 * c + 2]), lo(w[4 * c + 3]));
        } else {
          rh[c] = rl[c] = 0u;
        }
      }
      if (l == 0) {
        tmem_st16(trow + col8(kColW8, 0), rh);
        tmem_st16(trow + col8(kColWlo8, 0), rl);
      } else {
        tmem_st32(trow + col8(kColW8, l), rh);
        tmem_st32(trow + col8(kColWlo8, l), rl);
      }
    }
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const unsigned tD = tbase + kColSplitD + 64 * tg;                   // this group's accumulator
  const unsigned tDl = tD + ((unsigned)(q * 32) << 16) + 32 * hs;     // this thread's 32 columns
  const unsigned mbar = smem_u32(&S.mbar[tg]);
  // the group's operands: a_hi (BF16) and, in the second 16 KB, E5M2 copies of a and a_lo
  h16 *Bh = S.B[tg][0];
  unsigned char *B8 = reinterpret_cast<unsigned char *>(S.B[tg][1]);
  unsigned char *B8l = B8 + kMlpW * kSN;
  const unsigned aBh = smem_u32(Bh), aB8 = smem_u32(B8), aB8l = smem_u32(B8l);
  // after layer 4 the group's two buffers (contiguous) hold the FP32 activations
  // [feature][sample ^ (feature & 31)]
  float *h4 = reinterpret_cast<float *>(Bh);
  unsigned phase = 0;
  auto gsync = [&]() { asm volatile("bar.sync %0, %1;" ::"r"(1 + tg), "r"(kSGT) : "memory"); };
  // MN-major B (8 features x 8 samples core matrices): 128 B between sample groups, 1 KB
  // between feature groups; one 16-feature K step = 2 KB
  const unsigned idn = idesc_16(kSN, false, false, true);

  const long long ntiles = (in_count(in, n) + kSN - 1) / kSN;
  const long long tstride = (long long)gridDim.x * kSG;
  // the inputs of a group's next tile are read (threads gt < 64) while its current tile's
  // first layer runs on the tensor cores, off the tile's critical path
  long long nidx = 0;
  float nrh = 0.0f, nzh = 0.0f;
  bool nneed = false;
  const long long tile0 = (long long)blockIdx.x * kSG + tg;
  if (gt < kSN && tile0 < ntiles) nneed = tile_input(in, tile0 * kSN, gt, &nrh, &nzh, &nidx);
  for (long long tile = tile0; tile < ntiles; tile += tstride) {
    bool need = false;
    if (gt < kSN) {
      need = nneed;
      S.rh[tg][gt] = nrh;
      S.zh[tg][gt] = nzh;
      S.idx[tg][gt] = nidx;
      S.need[tg][gt] = need ? 1 : 0;
    }
    int any;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(any)
        : "r"((unsigned)need), "r"(1 + tg), "r"(kSGT)
        : "memory");
    if (!any) {  // nothing to evaluate in this tile: read the next tile's inputs and go on
      if (gt < kSN) {
        nneed = false;
        if (tile + tstride < ntiles)
          nneed = tile_input(in, (tile + tstride) * kSN, gt, &nrh, &nzh, &nidx);
      }
      continue;
    }
    {
      // Fourier features: direction j = gt % 32 for samples 8 (gt / 32) .. + 7 (range-reduced
      // phases, hardware sin / cos), sin into feature j and cos into feature 32 + j
      const int j = gt & 31, s0 = 8 * (gt >> 5);
      float sv[8], cv[8];
#pragma unroll
      for (int i = 0; i < 8; i++) {
        float ph = fmaf(S.Bf[j][0], S.rh[tg][s0 + i], S.Bf[j][1] * S.zh[tg][s0 + i]);
        ph -= rintf(ph);
        const float a = 6.283185307179586f * ph;
        sv[i] = __sinf(a);
        cv[i] = __cosf(a);
      }
      split_store8(Bh, B8, B8l, j, s0, sv);
      split_store8(Bh, B8, B8l, 32 + j, s0, cv);
    }
    proxy_fence();
    tc_fence_before();
    gsync();
    bool ok = true;
    for (int l = 0; l < 4 && ok; l++) {
      const int K = l == 0 ? kMlpF : kMlpW;
      if (gt == 0) {
        tc_fence_after();
        const unsigned aW = l == 0 ? smem_u32(S.W1) : smem_u32(S.Wh[l - 1]);
        const unsigned tW8 = tbase + col8(kColW8, l), tWl8 = tbase + col8(kColWlo8, l);
        const unsigned long long dW = mma_desc(aW, K);
        const unsigned long long dBh = mma_desc_mn(aBh, 128, 1024);
        // 8-bit MN-major B: 128 B between 16-sample groups, 512 B between feature groups;
        // one 32-feature K step = 2 KB
        const unsigned long long dB8 = mma_desc_mn(aB8, 128, 512);
        const unsigned long long dB8l = mma_desc_mn(aB8l, 128, 512);
        for (int k2 = 0; k2 < K / 32; k2++) {
          mma_bf16(tD, dW + 32u * k2, dBh + 256u * k2, idn, k2 > 0);       // W_hi a_hi
          mma_bf16(tD, dW + 32u * k2 + 16u, dBh + 256u * k2 + 128u, idn, 1);
          mma_f8_tmem_a(tD, tW8 + 8u * k2, dB8l + 128u * k2, idn, 1);      // W a_lo (E5M2)
          mma_f8_tmem_a(tD, tWl8 + 8u * k2, dB8 + 128u * k2, idn, 1);      // W_lo a (E5M2)
        }
        mma_commit(mbar);
      }
      if (l == 0 && gt < kSN) {
        nneed = false;
        if (tile + tstride < ntiles)
          nneed = tile_input(in, (tile + tstride) * kSN, gt, &nrh, &nzh, &nidx);
      }
      ok = mbar_wait(mbar, phase);
      phase ^= 1;
      tc_fence_after();
      if (!ok) {
        S.abort[tg] = 1;
        atomicExch(&g_mlp_error, 1);
      }
      if (ok) {
        float v[32];
        tmem_ld32(tDl, v);
        const float hb = 0.5f * S.bias[l][f];
#pragma unroll
        for (int i = 0; i < 32; i += 2) {
          // SiLU(z) = h (1 + tanh h), h = z / 2 = v/2 + b/2 (halving is exact), two columns
          // per packed instruction
          const float2 h = __ffma2_rn(make_float2(v[i], v[i + 1]), make_float2(0.5f, 0.5f),
                                      make_float2(hb, hb));
          float t0, t1;
          asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(h.x));
          asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(h.y));
          const float2 a = __ffma2_rn(h, make_float2(t0, t1), h);
          v[i] = a.x;
          v[i + 1] = a.y;
        }
        if (l < 3) {
#pragma unroll
          for (int c = 0; c < 2; c++) split_store16(Bh, B8, B8l, f, 32 * hs + 16 * c, v + 16 * c);
        } else {
          // the MMA of this layer has read the buffers: they now hold the FP32 activations
#pragma unroll
          for (int i = 0; i < 32; i++) h4[f * kSN + ((32 * hs + i) ^ lane)] = v[i];
        }
      }
      proxy_fence();
      tc_fence_before();
      gsync();
      ok = !S.abort[tg];
    }
    if (S.abort[tg]) break;
    {
      // output layer in FP32: thread gt -> sample gt % 64, inputs 32 (gt / 64) .. + 31, all
      // four outputs (W5T rows are broadcast; h4 reads are conflict-free by the swizzle);
      // then one thread per sample adds the four partial sums
      const int s = gt & (kSN - 1), kq = gt >> 6;
      float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 8
      for (int k = 32 * kq; k < 32 * kq + 32; k++) {
        const float h = h4[k * kSN + (s ^ (k & 31))];
        const float4 w = S.W5T[k];
        acc.x = fmaf(w.x, h, acc.x);
        acc.y = fmaf(w.y, h, acc.y);
        acc.z = fmaf(w.z, h, acc.z);
        acc.w = fmaf(w.w, h, acc.w);
      }
      // the partial sums replace h4 once every thread has read it
      float4 *red = reinterpret_cast<float4 *>(h4);  // [quarter][sample]
      gsync();
      red[kq * kSN + s] = acc;
      gsync();
      if (gt < kSN && S.need[tg][gt]) {
        const float4 a = red[gt], b = red[kSN + gt], c = red[2 * kSN + gt],
                     d = red[3 * kSN + gt];
        const float4 o = make_float4(S.bias5[0] + ((a.x + b.x) + (c.x + d.x)),
                                     S.bias5[1] + ((a.y + b.y) + (c.y + d.y)),
                                     S.bias5[2] + ((a.z + b.z) + (c.z + d.z)),
                                     S.bias5[3] + ((a.w + b.w) + (c.w + d.w)));
        reinterpret_cast<float4 *>(out)[S.idx[tg][gt]] = o;
      }
    }
    gsync();  // h4, the partial sums and the tile inputs are read before the next tile
  }
  // after a wait that ran out, let the MMA in flight finish (bounded) before the tensor
  // memory is released
  if (S.abort[tg] && gt == 0) mbar_wait(mbar, phase ^ 1);
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
  }
}

template <class In>
static int launch_mlp_split(const rt_mlp *m, const In &in, float *out, long long n,
                            cudaStream_t stream) {
  auto kern = mlp_split_kernel<In>;
  const size_t smem = sizeof(SplitSmem);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess)
    return set_error(RT_ECUDA, "mlp (split) smem attribute: %s", cudaGetErrorString(e));
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long tiles = (n + kSN - 1) / kSN;
  const long long groups = (tiles + kSG - 1) / kSG;
  const long long blocks = groups < nsm ? groups : nsm;
  kern<<<(unsigned)blocks, kSGT * kSG, smem, stream>>>(mlp_dev(m), in, out, n);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "mlp (split) launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

// FP16 operands: one pass; BF16 operands: the split three-pass product above.
template <class In>
static int launch_mlp(const rt_mlp *m, const In &in, float *out, long long n,
                      cudaStream_t stream) {
  if (n <= 0) return RT_OK;
  return m->precision == RT_MLP_BF16 ? launch_mlp_split<In>(m, in, out, n, stream)
                                     : launch_mlp_t<In, true>(m, in, out, n, stream);
}

// ---- list of the samples with gas (the rows the network needs) ----
// counts[pix] = samples of ray pix with gas
__global__ void gas_count_kernel(const __grid_constant__ MarchParams P, const Ray *__restrict__ rays,
                                 unsigned *__restrict__ counts) {
  const long long npix = (long long)P.nx * P.ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const Ray R = rays[pix];
  unsigned c = 0;
  if (R.hit)
    for (int k = 0; k < P.n_samples; k++) {
      bool gas;
      float rh, zh;
      sample_coords(P, R, k, &gas, &rh, &zh);
      c += gas ? 1u : 0u;
    }
  counts[pix] = c;
}

// In-place exclusive scan of 1024-element blocks; block totals to bsum.
__global__ void scan_block_kernel(unsigned *__restrict__ v, long long n, unsigned *__restrict__ bsum) {
  __shared__ unsigned warp_tot[32];
  const long long i = (long long)blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned x = i < n ? v[i] : 0u;
  unsigned incl = x;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    unsigned t = warp_tot[lane];
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  const unsigned before = (w > 0 ? warp_tot[w - 1] : 0u) + incl - x;
  if (i < n) v[i] = before;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = warp_tot[31];
}

// Exclusive scan of the nb block totals by one block (chunks of 1024), the grand total to
// *total; then every element gets its block's offset.
__global__ void scan_sums_kernel(unsigned *__restrict__ bsum, long long nb, unsigned *__restrict__ total) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long b0 = 0; b0 < nb; b0 += 1024) {
    const long long i = b0 + threadIdx.x;
    const unsigned x = i < nb ? bsum[i] : 0u;
    unsigned incl = x;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      unsigned t = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        unsigned y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const unsigned before = carry + (w > 0 ? warp_tot[w - 1] : 0u) + incl - x;
    if (i < nb) bsum[i] = before;
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// list[offset[pix] + j] = pix * n_samples + k for the j-th sample k of ray pix with gas
__global__ void gas_fill_kernel(const __grid_constant__ MarchParams P, const Ray *__restrict__ rays,
                                const unsigned *__restrict__ offsets,
                                const unsigned *__restrict__ boff, unsigned *__restrict__ list) {
  const long long npix = (long long)P.nx * P.ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pix >= npix) return;
  const Ray R = rays[pix];
  if (!R.hit) return;
  unsigned o = offsets[pix] + boff[pix / 1024];
  const unsigned base = (unsigned)(pix * P.n_samples);
  for (int k = 0; k < P.n_samples; k++) {
    bool gas;
    float rh, zh;
    sample_coords(P, R, k, &gas, &rh, &zh);
    if (gas) list[o++] = base + (unsigned)k;
  }
}

// Bytes of the sample-list buffers for n_pix rays of n_samples (0 when the sample index does
// not fit 32 bits: the network then runs over every sample).
size_t sample_list_bytes(long long npix, int n_samples) {
  const long long ns = npix * n_samples;
  if (npix <= 0 || ns >= (1LL << 32)) return 0;
  const long long nb = (npix + 1023) / 1024;
  return ((size_t)npix + (size_t)nb + 64 + (size_t)ns) * sizeof(unsigned);
}

struct SampleList {
  const unsigned *list = nullptr;
  const unsigned *count = nullptr;
};

// Layout of the list buffer: counts / offsets [npix], block sums [nb], total (64 words
// reserved), list [n_pix n_samples].
static SampleList sample_list_view(const MarchParams &P, const void *buf) {
  const long long npix = (long long)P.nx * P.ny;
  const long long nb = (npix + 1023) / 1024;
  const unsigned *total = reinterpret_cast<const unsigned *>(buf) + npix + nb;
  SampleList v;
  v.count = total;
  v.list = total + 64;
  return v;
}

static int build_sample_list(const MarchParams &P, const Ray *rays, void *buf, SampleList *out,
                             cudaStream_t stream) {
  const long long npix = (long long)P.nx * P.ny;
  const long long nb = (npix + 1023) / 1024;
  unsigned *counts = reinterpret_cast<unsigned *>(buf);
  unsigned *bsum = counts + npix;
  unsigned *total = bsum + nb;  // 64 words reserved
  unsigned *list = total + 64;
  gas_count_kernel<<<(unsigned)((npix + 127) / 128), 128, 0, stream>>>(P, rays, counts);
  scan_block_kernel<<<(unsigned)nb, 1024, 0, stream>>>(counts, npix, bsum);
  scan_sums_kernel<<<1, 1024, 0, stream>>>(bsum, nb, total);
  gas_fill_kernel<<<(unsigned)((npix + 127) / 128), 128, 0, stream>>>(P, rays, counts, bsum, list);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "sample list: %s", cudaGetErrorString(e));
  out->list = list;
  out->count = total;
  return RT_OK;
}

// Ray setups, the list of samples with gas (when list_buf is given) and the network outputs
// of those samples into mod ([pixel][sample] float4; other entries are left untouched).
int launch_mlp_rays(const rt_mlp *m, const MarchParams &P, float4 *mod, void *ray_buf,
                    void *list_buf, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  long long n = npix * P.n_samples;
  if (n == 0) return RT_OK;
  Ray *rays = reinterpret_cast<Ray *>(ray_buf);
  rays_kernel<<<(unsigned)((npix + 127) / 128), 128, 0, stream>>>(P, rays);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "ray setup launch: %s", cudaGetErrorString(e));
  if (list_buf) {
    SampleList sl;
    int rc = build_sample_list(P, rays, list_buf, &sl, stream);
    if (rc != RT_OK) return rc;
    ListInput in;
    in.P = P;
    in.rays = rays;
    in.list = sl.list;
    in.count = sl.count;
    return launch_mlp(m, in, reinterpret_cast<float *>(mod), n, stream);
  }
  RayInput in;
  in.P = P;
  in.rays = rays;
  return launch_mlp(m, in, reinterpret_cast<float *>(mod), n, stream);
}

size_t ray_buffer_bytes(long long npix) { return (size_t)npix * sizeof(Ray); }

int launch_rays(const MarchParams &P, Ray *rays, cudaStream_t stream) {
  const long long npix = (long long)P.nx * P.ny;
  if (npix == 0) return RT_OK;
  rays_kernel<<<(unsigned)((npix + 127) / 128), 128, 0, stream>>>(P, rays);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "ray setup launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

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


// ---------------------------------------------------------------------------------------
// Backward pass of the network: dL/dW and dL/db of every layer from per-sample dL/d(outputs)
// (reverse mode of the network written out by hand, on the tensor cores).
//
// The products are taken transposed, as in the split forward: features are the MMA's M (the
// TMEM lanes), samples its N. One persistent CTA per SM runs two tile groups of 64 samples
// (256 threads each: two per TMEM lane row, each owning 32 of the group's 64 accumulator
// columns), so that one group's epilogue arithmetic runs while the tensor core works on the
// other group's products. Tensor memory holds the weight-gradient accumulators dW2..dW4 (128
// columns each; zeroed at the start and shared by both groups) and a 64-column working
// accumulator per group. Shared memory holds the 16-bit weights (K-major core matrices, 112
// KB: the A operand of the forward products and, read MN-major, of the transposed ones) and per
// group three 16 KB operand buffers X, Y, D of core matrices of 8 features x 8 samples, which
// serve as MN-major B operands (features along K) and as K-major operands (samples along K)
// alike. With W_l mapping layer l-1 to layer l, a_0 = gamma the Fourier features, z_l the
// pre-activations and a_l = SiLU(z_l), per tile:
//   forward   z_l = W_l a_{l-1} + b_l for l = 1..4 (gamma in D, a_1 -> X, a_2 -> Y, a_3 -> X);
//             z_1..z_3 (16-bit) go to a per-CTA scratch in global memory (L2-resident);
//   output    on the CUDA cores in FP32, element by element in the layer-4 epilogue:
//             dW5 += delta_5 a_4^T and delta_4 = (W5^T delta_5) SiLU'(z_4) -> D, with
//             delta_5 = dL/d(outputs) scaled by a power of two that brings the largest below
//             one (FP16 has no room for raw gradients);
//   backward  l = 4, 3, 2: dW_l += delta_l a_{l-1}^T (M = out features, N = in features,
//             K = samples) and delta_{l-1} = (W_l^T delta_l) SiLU'(z_{l-1}) under one commit;
//             a_1 returns to X by a TMA bulk copy of the buffer's image, stored to the scratch
//             after layer 1 (a_3 overwrote it), and gamma is recomputed into Y;
//             dW1 = delta_1 gamma^T goes through the working columns and is summed in
//             registers.
// The inputs of a group's next tile are read during its first forward product. For a render,
// gather_list_kernel has packed the listed samples' inputs and output gradients in list
// order, so a tile's rows are two plain loads.
// The bias gradients are per-thread sums (a thread owns one feature row of the tile). Each
// group's first thread issues that group's MMAs; both groups accumulate into the same dW
// columns, so the order of the FP32 sums (not their terms) depends on the timing of the two.
// At the end each CTA adds its sums, unscaled, to the FP64 outputs with atomics. Waits on the
// mbarriers are bounded: on expiry the group records an error and stops, and the CTA releases
// its tensor memory after the MMAs in flight have finished.
// ---------------------------------------------------------------------------------------
constexpr int kBN = kSN;                  // samples per tile (MMA N): the layout of bmn_off
constexpr int kBG = 2;                    // tile groups per CTA
constexpr int kBGT = 256;                 // threads per group
constexpr int kBwdThreads = kBG * kBGT;
constexpr unsigned kColDW = 0;            // dW2, dW3, dW4: 128 columns each
constexpr unsigned kColBwdWork = 384;     // working accumulators: 64 columns per group

struct __align__(1024) BwdSmem {
  h16 W1[kMlpW * kMlpF];           // K-major core matrices (16 KB)
  h16 Wh[3][kMlpW * kMlpW];        // W2..W4 (96 KB)
  h16 buf[kBG][3][kMlpW * kBN];    // per group X, Y, D (16 KB each)
  float d5[kBG][4][kBN];           // scaled dL/d(outputs) of the group's samples
  float bias[4][kMlpW];
  float4 W5T[kMlpW];               // output layer, transposed: W5T[k] = W5[0..3][k]
  float rh[kBG][kBN], zh[kBG][kBN];
  float Bf[32][2];
  unsigned long long mbar[kBG];
  unsigned long long mbar_a1[kBG];  // bulk reload of a_1 into X
  unsigned tmem_base;
  int abort[kBG];
};
static_assert(sizeof(BwdSmem) <= 227 * 1024, "shared memory");
// per group in the scratch: z_1..z_3 (48 KB) and the image of the operand buffer holding a_1
constexpr size_t kBwdScratchU4 = 3 * 2 * 4 * kMlpW + kMlpW * kBN * sizeof(h16) / sizeof(uint4);
static_assert(kColBwdWork + 64 * kBG <= 512, "tensor memory");
// 96 columns of dW per warp (16 warps, four per lane quadrant) at zeroing and read-back
static_assert(kBwdThreads == 512 && 4 * 96 == kColBwdWork, "dW column split");

struct MlpGradsDev {
  double *dW[5];
  double *db[5];
};

// 8 values of feature k at samples s0..s0+7 (s0 multiple of 8), rounded to the 16-bit format,
// into an operand buffer of 8 features x 8 samples core matrices
template <bool F16>
__device__ __forceinline__ void store8s(h16 *B, int k, int s0, const float *v) {
  *reinterpret_cast<uint4 *>(B + bmn_off(k, s0)) =
      make_uint4(pack16<F16>(v[0], v[1]), pack16<F16>(v[2], v[3]), pack16<F16>(v[4], v[5]),
                 pack16<F16>(v[6], v[7]));
}

// SiLU'(z) of a pair, the arithmetic of dsilu() in packed two-lane instructions
__device__ __forceinline__ float2 dsilu2(float2 z) {
  const float2 h = __fmul2_rn(z, make_float2(0.5f, 0.5f));
  float t0, t1;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t0) : "f"(h.x));
  asm("tanh.approx.f32 %0, %1;" : "=f"(t1) : "f"(h.y));
  const float2 one = make_float2(1.0f, 1.0f);
  const float2 s = __ffma2_rn(make_float2(0.5f, 0.5f), make_float2(t0, t1), make_float2(0.5f, 0.5f));
  const float2 oms = __ffma2_rn(s, make_float2(-1.0f, -1.0f), one);  // 1 - s, one rounding
  return __fmul2_rn(s, __ffma2_rn(z, oms, one));
}

// 32-bit word i of four uint4 (i a compile-time constant after unrolling: no address taken,
// so the array stays in registers)
__device__ __forceinline__ unsigned word_of(const uint4 (&a)[4], int i) {
  const uint4 &u = a[i >> 2];
  return (i & 3) == 0 ? u.x : (i & 3) == 1 ? u.y : (i & 3) == 2 ? u.z : u.w;
}

// 8 packed pairs (16 values of feature k at samples s0..s0+15) into an operand buffer
__device__ __forceinline__ void store16p(h16 *B, int k, int s0, const unsigned *p) {
  *reinterpret_cast<uint4 *>(B + bmn_off(k, s0)) = make_uint4(p[0], p[1], p[2], p[3]);
  *reinterpret_cast<uint4 *>(B + bmn_off(k, s0 + 8)) = make_uint4(p[4], p[5], p[6], p[7]);
}

template <class In, bool F16>
__global__ void __launch_bounds__(kBwdThreads, 1)
    mlp_bwd_kernel(const MlpParamsDev Wp, const __grid_constant__ In in,
                   const float4 *__restrict__ gout, long long n,
                   const unsigned *__restrict__ gmax, h16 *__restrict__ spill,
                   const MlpGradsDev G) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  BwdSmem &S = *reinterpret_cast<BwdSmem *>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = tid / kBGT;           // tile group
  const int gt = tid % kBGT;          // thread within the group
  const int q = warp & 3;             // TMEM lane quadrant
  const int hs = (warp >> 2) & 1;     // half of the tile's samples (accumulator columns)
  const int f = q * 32 + lane;        // feature row (TMEM lane) of this thread

  // ---- one-time setup ----
  for (int i = tid; i < kMlpW * kMlpF; i += kBwdThreads)
    S.W1[cm_off(i / kMlpF, i % kMlpF, kMlpF)] = to16<F16>(Wp.W[0][i]);
  for (int l = 0; l < 3; l++)
    for (int i = tid; i < kMlpW * kMlpW; i += kBwdThreads)
      S.Wh[l][cm_off(i / kMlpW, i % kMlpW, kMlpW)] = to16<F16>(Wp.W[l + 1][i]);
  for (int i = tid; i < 4 * kMlpW; i += kBwdThreads) S.bias[i / kMlpW][i % kMlpW] = Wp.b[i / kMlpW][i % kMlpW];
  if (tid < 64) S.Bf[tid >> 1][tid & 1] = Wp.B[tid];
  if (tid == 0) {
    for (int i = 0; i < kBG; i++) {
      S.abort[i] = 0;
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar[i])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&S.mbar_a1[i])), "r"(1));
    }
  }
  for (int k = tid; k < kMlpW; k += kBwdThreads)
    S.W5T[k] = make_float4(Wp.W[4][k], Wp.W[4][kMlpW + k], Wp.W[4][2 * kMlpW + k],
                           Wp.W[4][3 * kMlpW + k]);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&S.tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  proxy_fence();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tbase = S.tmem_base;
  // zero the dW accumulators: warp w clears 96 columns of its lane quadrant
  const unsigned tq = tbase + ((unsigned)(q * 32) << 16);
  {
    unsigned zr[32];
#pragma unroll
    for (int j = 0; j < 32; j++) zr[j] = 0u;
#pragma unroll
    for (int c = 0; c < 3; c++) tmem_st32(tq + kColDW + 96 * (warp >> 2) + 32 * c, zr);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  const unsigned tD = tbase + kColBwdWork + 64 * g;              // this group's accumulator
  const unsigned tDl = tD + ((unsigned)(q * 32) << 16) + 32 * hs;  // this thread's 32 columns
  const unsigned mbar = smem_u32(&S.mbar[g]);
  h16 *X = S.buf[g][0], *Y = S.buf[g][1], *Dd = S.buf[g][2];
  const unsigned aX = smem_u32(X), aY = smem_u32(Y), aD = smem_u32(Dd);
  unsigned phase = 0;
  // power-of-two scale that brings the largest |dL/d(output)| below one
  int ex = 0;
  {
    const float gm = __uint_as_float(*gmax);
    if (gm > 0.0f && gm < 3.0e38f) frexpf(gm, &ex);
    ex = max(-120, min(120, ex));
  }
  const float scale = ldexpf(1.0f, -ex);
  float dw1[32];  // dW1[f][32 hs + j] of this group's tiles
#pragma unroll
  for (int j = 0; j < 32; j++) dw1[j] = 0.0f;
  float db[4] = {0.0f, 0.0f, 0.0f, 0.0f};   // db_1..db_4 of feature f over this thread's columns
  float dw5[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // dW5[o][f] over this thread's columns
  float db5[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // db_5 over a warp's samples (lane 0, gt < 64)
  // this group's pre-activations z_1..z_3: per (layer, column half, 8-sample quarter) a row
  // of 128 uint4 (one per feature), so a warp's stores are contiguous
  uint4 *Z = reinterpret_cast<uint4 *>(spill) + ((size_t)blockIdx.x * kBG + g) * kBwdScratchU4;
  uint4 *A1img = Z + 3 * 2 * 4 * kMlpW;  // 16 KB, 16-byte aligned
  const unsigned mbar_a1 = smem_u32(&S.mbar_a1[g]);
  unsigned a1_phase = 0;
  bool a1_pending = false;  // a reload of a_1 is in flight (issuing thread)
  auto zrow = [&](int l, int k) __attribute__((always_inline)) -> uint4 * { return Z + ((((l - 1) * 2 + hs) * 4 + k) * kMlpW + f); };

  auto gsync = [&]() __attribute__((always_inline)) { asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kBGT) : "memory"); };
  // group barrier that also returns whether any thread of the group passed p = true
  auto gsync_or = [&](bool p) __attribute__((always_inline)) -> bool {
    unsigned r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n"
        " bar.red.or.pred q, %2, %3, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((unsigned)p), "r"(1 + g), "r"(kBGT)
        : "memory");
    return r != 0;
  };
  bool last_ok = true;  // this thread's most recent wait ended in time
  auto wait_mma = [&]() __attribute__((always_inline)) -> bool {
    last_ok = mbar_wait(mbar, phase);
    if (last_ok) phase ^= 1;
    tc_fence_after();
    return last_ok;
  };
  // Fourier features of the tile's samples into features 0..63 of an operand buffer:
  // direction j = gt % 32 at samples 8 (gt / 32) .. + 7 (the arithmetic of features())
  auto write_features = [&](h16 *B) __attribute__((always_inline)) {
    const int j = gt & 31, s0 = 8 * (gt >> 5);
    float sv[8], cv[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
      float ph = fmaf(S.Bf[j][0], S.rh[g][s0 + i], S.Bf[j][1] * S.zh[g][s0 + i]);
      ph -= rintf(ph);
      const float a = 6.283185307179586f * ph;
      sv[i] = __sinf(a);
      cv[i] = __cosf(a);
    }
    store8s<F16>(B, j, s0, sv);
    store8s<F16>(B, 32 + j, s0, cv);
  };

  // ---- MMA issue (the group's first thread) ----
  // forward z_l: A = W_l (K-major), B = a_{l-1} (MN-major: 128 B between sample groups, 1 KB
  // between feature groups, 2 KB per 16-feature K step)
  auto issue_forward = [&](int l, unsigned ain) __attribute__((always_inline)) {
    const int K = l == 1 ? kMlpF : kMlpW;
    const unsigned aW = l == 1 ? smem_u32(S.W1) : smem_u32(S.Wh[l - 2]);
    const unsigned long long dA = mma_desc(aW, K), dB = mma_desc_mn(ain, 128, 1024);
    const unsigned id = idesc_16(kBN, F16, false, true);
    for (int ks = 0; ks < K / 16; ks++) mma_bf16(tD, dA + 16u * ks, dB + 128u * ks, id, ks > 0);
    mma_commit(mbar);
  };
  // backward step l: dW_l += delta_l a_{l-1}^T (A = delta_l from D and B = a_{l-1}, both with
  // the samples along K: K-major, 1 KB between feature groups), then W_l^T delta_l into the
  // working columns (A = W_l read MN-major: 128 B between input-feature groups, 2 KB between
  // output-feature groups; B = delta_l MN-major)
  auto issue_backward = [&](int l, unsigned ax) __attribute__((always_inline)) {
    const unsigned long long dA = mma_desc(aD, kBN), dX = mma_desc(ax, kBN);
    const unsigned idw = idesc_16(kMlpW, F16, false, false);
    const unsigned tW = tbase + kColDW + 128u * (unsigned)(l - 2);
    for (int ks = 0; ks < kBN / 16; ks++) mma_bf16(tW, dA + 16u * ks, dX + 16u * ks, idw, 1);
    const unsigned long long dWt = mma_desc_mn(smem_u32(S.Wh[l - 2]), 128, 2048);
    const unsigned long long dDl = mma_desc_mn(aD, 128, 1024);
    const unsigned idt = idesc_16(kBN, F16, true, true);
    for (int ks = 0; ks < kMlpW / 16; ks++)
      mma_bf16(tD, dWt + 256u * ks, dDl + 128u * ks, idt, ks > 0);
    mma_commit(mbar);
  };
  // dW1 of the tile: delta_1 gamma^T into the working columns (gamma in Y, N = 64)
  auto issue_dw1 = [&]() __attribute__((always_inline)) {
    const unsigned long long dA = mma_desc(aD, kBN), dG = mma_desc(aY, kBN);
    const unsigned id = idesc_16(kMlpF, F16, false, false);
    for (int ks = 0; ks < kBN / 16; ks++) mma_bf16(tD, dA + 16u * ks, dG + 16u * ks, id, ks > 0);
    mma_commit(mbar);
  };

  bool bad = false;  // group-uniform: a wait ran out
  const long long ntiles = (in_count(in, n) + kBN - 1) / kBN;
  const long long tstride = (long long)gridDim.x * kBG;
  const long long tile0 = (long long)blockIdx.x * kBG + g;
  // inputs of the group's next tile (threads gt < 64), read a tile ahead so that the list and
  // ray lookups stay off the tile's chain of dependent phases
  float nrh = 0.0f, nzh = 0.0f;
  float4 nd = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  bool nneed = false;
  auto fetch = [&](long long t) __attribute__((always_inline)) {
    nneed = false;
    nrh = nzh = 0.0f;
    nd = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (gt < kBN && t < ntiles) {
      long long s = 0;
      nneed = tile_input(in, t * kBN, gt, &nrh, &nzh, &s);
      if (nneed) nd = gout[s];  // scaled when stored: nothing here waits for the load
    }
  };
  fetch(tile0);
  for (long long tile = tile0; tile < ntiles; tile += tstride) {
    // ---- inputs: sample coordinates and scaled output gradients ----
    const bool need = nneed;
    if (gt < kBN) {
      const float4 d = make_float4(nd.x * scale, nd.y * scale, nd.z * scale, nd.w * scale);
      S.rh[g][gt] = nrh;
      S.zh[g][gt] = nzh;
      S.d5[g][0][gt] = d.x;
      S.d5[g][1][gt] = d.y;
      S.d5[g][2][gt] = d.z;
      S.d5[g][3][gt] = d.w;
      float r[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
      for (int o = 0; o < 4; o++)
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) r[o] += __shfl_xor_sync(0xffffffffu, r[o], off);
      if (lane == 0)
#pragma unroll
        for (int o = 0; o < 4; o++) db5[o] += r[o];
    }
    if (!gsync_or(need)) {  // no sample of this tile needs the network
      fetch(tile + tstride);
      continue;
    }
    write_features(Dd);
    proxy_fence();
    tc_fence_before();
    gsync();

    // ---- forward: a_1 -> X, a_2 -> Y, a_3 -> X; layer 4 ends in the output layer ----
#pragma unroll
    for (int l = 1; l <= 4; l++) {
      if (gt == 0) {
        tc_fence_after();
        issue_forward(l, l == 1 ? aD : (l == 3 ? aY : aX));
        if (l == 2) {  // keep an image of a_1 (X): a_3 overwrites it, dW2 needs it again
          asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(A1img),
                       "r"(aX), "r"(kMlpW * kBN * (int)sizeof(h16))
                       : "memory");
          asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
      }
      if (l == 1) fetch(tile + tstride);
      const bool ok = wait_mma();
      if (ok) {
        const float b = S.bias[l - 1][f];
        const float2 b2 = make_float2(b, b);
        if (l < 4) {
          h16 *Aout = l == 2 ? Y : X;
          float v[32];
          tmem_ld32(tDl, v);
#pragma unroll
          for (int h = 0; h < 2; h++) {
            unsigned zp[8], ap[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const float2 z = __fadd2_rn(make_float2(v[16 * h + 2 * j], v[16 * h + 2 * j + 1]), b2);
              zp[j] = pack16<F16>(z.x, z.y);
              ap[j] = silu2p<F16>(zp[j]);
            }
            *zrow(l, 2 * h) = make_uint4(zp[0], zp[1], zp[2], zp[3]);
            *zrow(l, 2 * h + 1) = make_uint4(zp[4], zp[5], zp[6], zp[7]);
            store16p(Aout, f, 32 * hs + 16 * h, ap);
          }
        } else {
          // output layer (FP32, pairs of samples): dW5 += delta_5 a_4^T and
          // delta_4 = (W5^T delta_5) SiLU'(z_4)
          float2 dsum = make_float2(0.0f, 0.0f);
          float2 acc5[4] = {dsum, dsum, dsum, dsum};
          const float4 w5 = S.W5T[f];  // W5 column of this thread's feature (FP32)
          const float2 w5x = make_float2(w5.x, w5.x), w5y = make_float2(w5.y, w5.y);
          const float2 w5z = make_float2(w5.z, w5.z), w5w = make_float2(w5.w, w5.w);
          float v[32];
          tmem_ld32(tDl, v);
#pragma unroll
          for (int h = 0; h < 2; h++) {
            unsigned dp[8];
#pragma unroll
            for (int j = 0; j < 8; j++) {
              const int sc = 32 * hs + 16 * h + 2 * j;
              const float2 zf = __fadd2_rn(make_float2(v[16 * h + 2 * j], v[16 * h + 2 * j + 1]), b2);
              const unsigned zp = pack16<F16>(zf.x, zf.y);
              const float2 a = unpack16<F16>(silu2p<F16>(zp));
              const float2 z = unpack16<F16>(zp);
              const float2 dx = *reinterpret_cast<const float2 *>(&S.d5[g][0][sc]);
              const float2 dy = *reinterpret_cast<const float2 *>(&S.d5[g][1][sc]);
              const float2 dz = *reinterpret_cast<const float2 *>(&S.d5[g][2][sc]);
              const float2 dw = *reinterpret_cast<const float2 *>(&S.d5[g][3][sc]);
              acc5[0] = __ffma2_rn(dx, a, acc5[0]);
              acc5[1] = __ffma2_rn(dy, a, acc5[1]);
              acc5[2] = __ffma2_rn(dz, a, acc5[2]);
              acc5[3] = __ffma2_rn(dw, a, acc5[3]);
              const float2 t =
                  __ffma2_rn(w5x, dx, __ffma2_rn(w5y, dy, __ffma2_rn(w5z, dz, __fmul2_rn(w5w, dw))));
              const float2 dl = __fmul2_rn(t, dsilu2(z));
              dsum = __fadd2_rn(dsum, dl);
              dp[j] = pack16<F16>(dl.x, dl.y);
            }
            store16p(Dd, f, 32 * hs + 16 * h, dp);
          }
#pragma unroll
          for (int o = 0; o < 4; o++) dw5[o] += acc5[o].x + acc5[o].y;
          db[3] += dsum.x + dsum.y;
        }
      }
      if (l == 2 && gt == 0)  // the image is read out before layer 3 writes a_3 into X
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      proxy_fence();
      tc_fence_before();
      bad = gsync_or(!ok);
      if (bad) break;
    }
    if (bad) break;

    // ---- backward steps l = 4, 3, 2: a_{l-1} is a_3 (X), a_2 (Y), a_1 (X, recomputed) ----
#pragma unroll
    for (int l = 4; l >= 2; l--) {
      uint4 zq[4];  // z_{l-1} of this thread
#pragma unroll
      for (int k = 0; k < 4; k++) zq[k] = *zrow(l - 1, k);
      bool a1_ok = true;
      if (gt == 0) {
        if (l == 2) {  // a_1 back in X
          a1_ok = mbar_wait(mbar_a1, a1_phase);
          if (a1_ok) {
            a1_phase ^= 1;
            a1_pending = false;
          }
        }
        tc_fence_after();
        if (a1_ok) issue_backward(l, l == 3 ? aY : aX);  // else the group's wait runs out
      }
      const bool ok = wait_mma();
      if (ok && l == 4 && gt == 0) {  // dW4 has read a_3: reload a_1 into X
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar_a1),
                     "r"(kMlpW * kBN * (int)sizeof(h16))
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(aX),
            "l"(A1img), "r"(kMlpW * kBN * (int)sizeof(h16)), "r"(mbar_a1)
            : "memory");
        a1_pending = true;
      }
      if (ok) {
        float2 dsum = make_float2(0.0f, 0.0f);
        float v[32];
        tmem_ld32(tDl, v);
#pragma unroll
        for (int h = 0; h < 2; h++) {
          unsigned dp[8];
#pragma unroll
          for (int j = 0; j < 8; j++) {
            const float2 z = unpack16<F16>(word_of(zq, 8 * h + j));
            const float2 d = __fmul2_rn(make_float2(v[16 * h + 2 * j], v[16 * h + 2 * j + 1]), dsilu2(z));
            dsum = __fadd2_rn(dsum, d);
            dp[j] = pack16<F16>(d.x, d.y);
          }
          store16p(Dd, f, 32 * hs + 16 * h, dp);  // delta_l has been read
        }
        db[l - 2] += dsum.x + dsum.y;
        if (l == 2) write_features(Y);  // gamma for dW1 (a_2 has been read)
      }
      proxy_fence();
      tc_fence_before();
      bad = gsync_or(!ok);
      if (bad) break;
    }
    if (bad) break;

    // ---- dW1 += delta_1 gamma^T, through the working columns ----
    if (gt == 0) {
      tc_fence_after();
      issue_dw1();
    }
    const bool ok = wait_mma();
    if (ok) {
      float v[32];
      tmem_ld32(tDl, v);
#pragma unroll
      for (int j = 0; j < 32; j++) dw1[j] += v[j];
    }
    tc_fence_before();
    bad = gsync_or(!ok);  // the tile's buffers and inputs are free after this barrier
    if (bad) break;
  }

  if (bad) {
    if (!last_ok) atomicExch(&g_mlp_error, 1);
    if (gt == 0) {
      S.abort[g] = 1;
      // let an MMA and a bulk copy still in flight finish (bounded) before the tensor memory
      // and the shared memory are released
      if (!last_ok) mbar_wait(mbar, phase);
      if (a1_pending) mbar_wait(mbar_a1, a1_phase);
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!S.abort[0] && !S.abort[1]) {
    const double un = ldexp(1.0, ex);
#pragma unroll
    for (int j = 0; j < 32; j++)
      atomicAdd(G.dW[0] + f * kMlpF + 32 * hs + j, (double)dw1[j] * un);
#pragma unroll
    for (int l = 0; l < 4; l++) atomicAdd(G.db[l] + f, (double)db[l] * un);
#pragma unroll
    for (int o = 0; o < kMlpOut; o++) atomicAdd(G.dW[4] + o * kMlpW + f, (double)dw5[o] * un);
    if (gt < kBN && lane == 0)
#pragma unroll
      for (int o = 0; o < kMlpOut; o++) atomicAdd(G.db[4] + o, (double)db5[o] * un);
    // dW2..dW4: warp w reads 96 columns of its lane quadrant (16-column chunks never straddle
    // a layer boundary)
    for (int c = 0; c < 6; c++) {
      const int col = 96 * (warp >> 2) + 16 * c;
      float v[16];
      tmem_ld16(tq + kColDW + col, v);
      double *dst = G.dW[1 + col / kMlpW] + f * kMlpW + col % kMlpW;
#pragma unroll
      for (int j = 0; j < 16; j++) atomicAdd(dst + j, (double)v[j] * un);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(512));
  }
}

// max |x| over n float4 values into *out (float bits; out zeroed by the caller)
__global__ void absmax_kernel(const float4 *__restrict__ x, long long n, unsigned *out) {
  float m = 0.0f;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float4 v = x[i];
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0 && m > 0.0f) atomicMax(out, __float_as_uint(m));
}

// pre-activation scratch of the backward kernel: z_1..z_3 of one tile per group and CTA
static size_t mlp_spill_bytes(long long blocks) {
  return (size_t)blocks * kBG * kBwdScratchU4 * sizeof(uint4);
}

// Zeroes the gradient outputs and runs the backward kernel over n samples; spill must hold
// mlp_spill_bytes(blocks) with blocks = mlp_bwd_blocks(n).
static long long mlp_bwd_blocks(long long n) {
  int dev = 0, nsm = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const long long pairs = ((n + kBN - 1) / kBN + kBG - 1) / kBG;
  return pairs < nsm ? (pairs > 0 ? pairs : 1) : nsm;
}

template <class In, bool F16>
static int launch_mlp_bwd_t(const rt_mlp *m, const In &in, const float4 *gout, long long n,
                            const unsigned *gmax, h16 *spill, const rt_mlp_grads *g,
                            cudaStream_t stream) {
  auto kern = mlp_bwd_kernel<In, F16>;
  const size_t smem = sizeof(BwdSmem);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess)
    return set_error(RT_ECUDA, "mlp backward smem attribute: %s", cudaGetErrorString(e));
  const int din[5] = {kMlpF, kMlpW, kMlpW, kMlpW, kMlpW};
  const int dout[5] = {kMlpW, kMlpW, kMlpW, kMlpW, kMlpOut};
  MlpGradsDev G;
  for (int l = 0; l < 5; l++) {
    G.dW[l] = g->dW[l];
    G.db[l] = g->db[l];
    e = cudaMemsetAsync(g->dW[l], 0, sizeof(double) * din[l] * dout[l], stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(g->db[l], 0, sizeof(double) * dout[l], stream);
    if (e != cudaSuccess) return set_error(RT_ECUDA, "gradient memset: %s", cudaGetErrorString(e));
  }
  if (n <= 0) return RT_OK;
  kern<<<(unsigned)mlp_bwd_blocks(n), kBwdThreads, smem, stream>>>(mlp_dev(m), in, gout, n, gmax,
                                                                   spill, G);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "mlp backward launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

template <class In>
static int launch_mlp_bwd(const rt_mlp *m, const In &in, const float4 *gout, long long n,
                          const unsigned *gmax, h16 *spill, const rt_mlp_grads *g,
                          cudaStream_t stream) {
  return m->precision == RT_MLP_BF16
             ? launch_mlp_bwd_t<In, false>(m, in, gout, n, gmax, spill, g, stream)
             : launch_mlp_bwd_t<In, true>(m, in, gout, n, gmax, spill, g, stream);
}

int mlp_grads_validate(const rt_mlp_grads *g) {
  if (!g) return set_error(RT_EINVAL, "null network gradients");
  for (int l = 0; l < 5; l++)
    if (!g->dW[l] || !g->db[l])
      return set_error(RT_EINVAL, "null weight or bias gradient of layer %d", l);
  return RT_OK;
}

size_t mlp_bwd_scratch_bytes(long long n) { return mlp_spill_bytes(mlp_bwd_blocks(n)); }

// Backward pass over the samples of a render (rays from the forward's pre-pass in ray_buf,
// per-sample dL/d(outputs) in dmod, their largest magnitude in *dmax).
// Inputs and output gradients of the listed samples in list order, padded with zeros to whole
// backward tiles: xy[i] = (rhat, zhat) of sample list[i], g[i] = dmod[list[i]] (zero without
// gas); i < *count rounded up to a multiple of 64.
__global__ void gather_list_kernel(const __grid_constant__ MarchParams P,
                                   const Ray *__restrict__ rays, const unsigned *__restrict__ list,
                                   const unsigned *__restrict__ count,
                                   const float4 *__restrict__ dmod, float2 *__restrict__ xy,
                                   float4 *__restrict__ g) {
  const long long c = *count;
  const long long cp = (c + kBN - 1) / kBN * kBN;
  const unsigned ns = (unsigned)P.n_samples;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < cp;
       i += (long long)gridDim.x * blockDim.x) {
    float rh = 0.0f, zh = 0.0f;
    float4 d = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (i < c) {
      const unsigned v = list[i];
      bool gas;
      sample_coords(P, rays[v / ns], (int)(v % ns), &gas, &rh, &zh);
      if (gas) d = dmod[v];
    }
    xy[i] = make_float2(rh, zh);
    g[i] = d;
  }
}

size_t mlp_bwd_gather_entries(long long n) { return (size_t)((n + kBN - 1) / kBN * kBN); }

int launch_mlp_bwd_rays(const rt_mlp *m, const MarchParams &P, const void *ray_buf,
                        const void *list_buf, const float4 *dmod, const unsigned *dmax,
                        void *spill, float2 *xy_buf, float4 *g_buf, const rt_mlp_grads *g,
                        cudaStream_t stream) {
  long long n = (long long)P.nx * P.ny * P.n_samples;
  if (list_buf) {
    const SampleList sl = sample_list_view(P, list_buf);
    if (n > 0) {
      const long long nb = (n + 255) / 256;
      gather_list_kernel<<<(unsigned)(nb < 148 * 16 ? nb : 148 * 16), 256, 0, stream>>>(
          P, reinterpret_cast<const Ray *>(ray_buf), sl.list, sl.count, dmod, xy_buf, g_buf);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return set_error(RT_ECUDA, "gather launch: %s", cudaGetErrorString(e));
    }
    PackedInput in;
    in.xy = xy_buf;
    in.count = sl.count;
    return launch_mlp_bwd(m, in, g_buf, n, dmax, reinterpret_cast<h16 *>(spill), g, stream);
  }
  RayInput in;
  in.P = P;
  in.rays = reinterpret_cast<const Ray *>(ray_buf);
  return launch_mlp_bwd(m, in, dmod, n, dmax, reinterpret_cast<h16 *>(spill), g, stream);
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

// Backward pass at explicit inputs (see rt.h).
extern "C" int rt_mlp_backward(const rt_mlp *mlp, const float *xy, const float *dout,
                               long long n, const rt_mlp_grads *grads, void *stream) {
  using namespace rtb;
  int rc = mlp_check(mlp);
  if (rc == RT_OK) rc = mlp_grads_validate(grads);
  if (rc == RT_OK && n < 0) rc = set_error(RT_EINVAL, "negative point count");
  if (rc == RT_OK && n > 0 && (!xy || !dout)) rc = set_error(RT_EINVAL, "null inputs");
  if (rc != RT_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long blocks = mlp_bwd_blocks(n);
  const size_t sp = mlp_spill_bytes(blocks);
  char *buf = nullptr;
  cudaError_t e = stream_alloc((void **)&buf, sp + 256, st);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "mlp backward scratch (%zu bytes): %s", sp + 256,
                     cudaGetErrorString(e));
  unsigned *gmax = reinterpret_cast<unsigned *>(buf + sp);
  e = cudaMemsetAsync(gmax, 0, sizeof(unsigned), st);
  if (e == cudaSuccess && n > 0) {
    long long nb = (n + 255) / 256;
    absmax_kernel<<<(unsigned)(nb < 1184 ? nb : 1184), 256, 0, st>>>(
        reinterpret_cast<const float4 *>(dout), n, gmax);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    rc = set_error(RT_ECUDA, "gradient scale: %s", cudaGetErrorString(e));
  } else {
    XYInput in;
    in.xy = xy;
    in.n = n;
    rc = launch_mlp_bwd(mlp, in, reinterpret_cast<const float4 *>(dout), n, gmax,
                        reinterpret_cast<h16 *>(buf), grads, st);
  }
  cudaFreeAsync(buf, st);
  if (rc == RT_OK) clear_error();
  return rc;
}
