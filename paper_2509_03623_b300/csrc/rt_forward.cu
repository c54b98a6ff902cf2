// Forward march kernel.
//
// Mapping: a warp marches R = 32/LPR neighbouring rays at a time (one work unit); the LPR
// lanes of a ray split its channels (lane q holds channels q, q+LPR, ... in registers, CPL
// of them). The grid is persistent (one wave) and work units are interleaved over its warps;
// the double-precision ray setups (chord through the bounding cylinder) of 32 rays are
// computed at once, one per lane, and kept in shared memory. Samples advance in batches of
// LPR: in the physics phase lane q evaluates the channel-independent physics of sample kb+q
// of its ray (fields, CO layer, Keplerian velocity, line width, LTE source and opacity) once
// and publishes it in shared memory; batches without gas on any ray are skipped (warp vote);
// in the channel phase every lane walks the batch's samples in order (fully unrolled),
// evaluating the Doppler-shifted Gaussian profile and advancing optical depth, transmittance
// and intensity front to back (Eq. rt-int with Eq. optical_depth; the source is constant
// over each segment).
//
// Per sample-channel evaluation: 7 FP32 operations and 2 MUFU.EX2. The optical depth is
// summed per batch and folded into a per-channel base at the end of every batch (blocked
// summation: about 2 N_s / LPR roundings instead of N_s).
#include <mutex>

#include "rt_internal.cuh"

namespace rtb {

constexpr int kWarps = 4;  // warps per block

// Channel-independent physics of sample k of a ray: {kd, a, b, S} with
//   kd  optical depth per unit profile (log2 units): dtau_c = kd 2^{-d_c^2}, 0 without gas
//   a,b profile argument d_c = v_c b - a (b = sqrt(log2 e)/alpha, a = v_los b)
//   S   LTE source function in units of 2 h nu0^3 / c^2
__device__ __forceinline__ float4 sample_physics(const MarchParams &P, const float *tab,
                                                 const Ray &R, int k) {
  float kf = (float)k;
  float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
  float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
  float r2 = fmaf(R.x, R.x, y * y);
  Cell c = locate(P, z, r2);
  float4 out = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
  if (!(c.gas && R.hit && k < P.n_samples)) return out;
  float T = bilerp(P.T, P.nr, c);
  float n = bilerp(P.n, P.nr, c);
  float vt = bilerp(P.vt, P.nr, c);
  const float *hl = P.hlo + c.i0;
  const float *hh = P.hhi + c.i0;
  float hlo = lerpf(__ldg(hl), __ldg(hl + 1), c.fr);
  float hhi = lerpf(__ldg(hh), __ldg(hh + 1), c.fr);
  float X;
  if (P.hard_edge) {
    X = (c.zr >= hlo && c.zr <= hhi) ? P.x_co : 0.0f;
  } else {
    float ea = ex2((hlo - c.zr) * P.edge_k);
    float eb = ex2((c.zr - hhi) * P.edge_k);
    X = P.x_co * rcp((1.0f + ea) * (1.0f + eb));
  }
  // Keplerian rotation: v_los = sqrt(GM) sin i x (r^2 + z^2)^{-3/4} + v_sys
  float vlos = fmaf(R.vfac, kepler_q(fmaf(z, z, r2)), P.vsys);
  // line width
  float Tg = fmaxf(T, 1e-3f);
  float a2 = P.vturb_mach ? Tg * fmaf(P.c_mach, vt * vt, P.c_th) : fmaf(P.c_th, Tg, vt * vt);
  float ia = rsq(a2);
  // LTE: source function and tabulated lower-level opacity factor
  float phi = lte_phi(tab, lg2(Tg), nullptr);
  float eS = ex2(-P.theta_s * rcp(Tg));
  out.w = eS * rcp(1.0f - eS);
  out.x = P.kappa_k * (X * n) * ex2(phi) * ia * R.ds;
  out.z = ia * 1.2011224087864498f;  // b = sqrt(log2 e) / alpha
  out.y = vlos * out.z;              // a = v_los b
  return out;
}

template <int LPR, int CPL, bool UNIF>
__global__ void __launch_bounds__(kWarps * 32)
    march_fwd_kernel(const __grid_constant__ MarchParams P, float *__restrict__ cube) {
  constexpr int R = 32 / LPR;  // rays marched together by one warp (one work unit)
  constexpr int G = 32 / R;    // work units whose ray setups are computed together
  __shared__ __align__(16) float s_tab[kTabSeg * 4];
  __shared__ float4 s_ph[kWarps][32];
  __shared__ Ray s_ray[kWarps][32];
  for (int i = threadIdx.x; i < kTabSeg * 4; i += blockDim.x) s_tab[i] = P.tab[i];
  __syncthreads();

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = lane % LPR, rr = lane / LPR;
  const long long npix = (long long)P.nx * P.ny;
  const long long nunits = (npix + R - 1) / R;
  const long long W = (long long)gridDim.x * kWarps;  // warps in the grid
  float4 *ph = s_ph[wib];

  float vr[UNIF ? 1 : CPL];
  if (!UNIF) {
#pragma unroll
    for (int j = 0; j < CPL; j++) vr[j] = P.v[min(q + LPR * j, RT_MAX_CH - 1)];
  }
  const float vq = P.v0 + (float)q * P.dv;  // velocity of this lane's first channel
  const float dvs = (float)LPR * P.dv;      // spacing between this lane's channels

  // Work units u = gw, gw + W, gw + 2W, ... (interleaved over the grid for balance); the
  // setups of G units (32 rays) are computed at once, one ray per lane.
  for (long long u0 = (long long)blockIdx.x * kWarps + wib; u0 < nunits; u0 += W * G) {
    {
      long long pix = (u0 + (long long)(lane / R) * W) * R + lane % R;
      bool act = pix < npix;
      Ray s = setup_ray(P, act ? (int)(pix % P.nx) : 0, act ? (int)(pix / P.nx) : 0, act);
      __syncwarp();
      s_ray[wib][lane] = s;
      __syncwarp();
    }
    for (int g = 0; g < G; g++) {
      const long long u = u0 + (long long)g * W;
      if (u >= nunits) break;
      const long long pix = u * R + rr;
      const Ray ray = s_ray[wib][g * R + rr];
      float tl[CPL], tb[CPL], Tr[CPL], I[CPL];
#pragma unroll
      for (int j = 0; j < CPL; j++) {
        tl[j] = 0.0f;
        tb[j] = 0.0f;
        Tr[j] = 1.0f;
        I[j] = 0.0f;
      }
      const int nsamp = __any_sync(0xffffffffu, ray.hit) ? P.n_samples : 0;
      for (int kb = 0; kb < nsamp; kb += LPR) {
        const float4 mine = sample_physics(P, s_tab, ray, kb + q);
        if (!__any_sync(0xffffffffu, mine.x > 0.0f)) continue;  // no gas in this batch
        ph[lane] = mine;
        __syncwarp();
        // every sample of the batch in order; samples without gas are exact no-ops
#pragma unroll
        for (int t = 0; t < LPR; t++) {
          const float4 p = ph[rr * LPR + t];  // kd, a, b, S of sample kb+t of this ray
          const float dc = fmaf(vq, p.z, -p.y), db = dvs * p.z;
#pragma unroll
          for (int j = 0; j < CPL; j++) {
            float d = UNIF ? fmaf((float)j, db, dc) : fmaf(vr[j], p.z, -p.y);
            tl[j] = fmaf(p.x, ex2(d * -d), tl[j]);
            float Tn = ex2(-tb[j] - tl[j]);
            I[j] = fmaf(p.w, Tr[j] - Tn, I[j]);
            Tr[j] = Tn;
          }
        }
#pragma unroll
        for (int j = 0; j < CPL; j++) {
          tb[j] += tl[j];
          tl[j] = 0.0f;
        }
        __syncwarp();
      }
      if (pix < npix) {
#pragma unroll
        for (int j = 0; j < CPL; j++) {
          int ch = q + LPR * j;
          if (ch < P.nch) cube[(long long)ch * npix + pix] = fmaf(I[j], P.out_scale, P.I0 * Tr[j]);
        }
      }
    }
  }
}

// Blocks of a kernel resident on the whole device at once (queried once per kernel and
// device, then cached).
static int resident_blocks(const void *kernel) {
  struct Entry {
    const void *k;
    int dev, blocks;
  };
  static std::mutex mu;
  static Entry cache[64];
  static int n = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n; i++)
      if (cache[i].k == kernel && cache[i].dev == dev) return cache[i].blocks;
  }
  int nb = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, kWarps * 32, 0) != cudaSuccess ||
      nb < 1)
    nb = 1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 1;
  std::lock_guard<std::mutex> lk(mu);
  if (n < 64) cache[n++] = Entry{kernel, dev, nb * nsm};
  return nb * nsm;
}

template <int LPR, int CPL, bool UNIF>
static void launch_t(const MarchParams &P, float *cube, cudaStream_t stream) {
  auto kern = march_fwd_kernel<LPR, CPL, UNIF>;
  long long npix = (long long)P.nx * P.ny;
  long long units = (npix + (32 / LPR) - 1) / (32 / LPR);
  long long need = (units + kWarps - 1) / kWarps;
  long long cap = resident_blocks((const void *)kern);
  long long blocks = need < cap ? need : cap;
  kern<<<(unsigned)blocks, kWarps * 32, 0, stream>>>(P, cube);
}

template <int LPR, int CPL>
static void launch_u(const MarchParams &P, float *cube, cudaStream_t stream) {
  if (P.v_uniform)
    launch_t<LPR, CPL, true>(P, cube, stream);
  else
    launch_t<LPR, CPL, false>(P, cube, stream);
}

// Channels per lane (4, or 8 above 128 channels) and lanes per ray (power of two).
void lane_layout(int nch, int *lpr, int *cpl) {
  int c = nch > 128 ? 8 : 4;
  int need = (nch + c - 1) / c, l = 1;
  while (l < need) l *= 2;
  *lpr = l;
  *cpl = c;
}

int launch_forward(const MarchParams &P, float *cube, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return RT_OK;
  int LPR, CPL;
  lane_layout(P.nch, &LPR, &CPL);
  if (CPL == 8) launch_u<32, 8>(P, cube, stream);
  else if (LPR == 32) launch_u<32, 4>(P, cube, stream);
  else if (LPR == 16) launch_u<16, 4>(P, cube, stream);
  else if (LPR == 8) launch_u<8, 4>(P, cube, stream);
  else if (LPR == 4) launch_u<4, 4>(P, cube, stream);
  else if (LPR == 2) launch_u<2, 4>(P, cube, stream);
  else launch_u<1, 4>(P, cube, stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "forward launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

// Work count: (ray, sample) pairs of hit rays that fall inside the gas grid, i.e. the
// executed (rather than nominal) samples of a render.
__global__ void count_gas_kernel(const __grid_constant__ MarchParams P,
                                 unsigned long long *__restrict__ count) {
  const long long npix = (long long)P.nx * P.ny;
  const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long n = 0;
  if (pix < npix) {
    Ray R = setup_ray(P, (int)(pix % P.nx), (int)(pix / P.nx), true);
    if (R.hit) {
      for (int k = 0; k < P.n_samples; k++) {
        float kf = (float)k;
        float y = sample_coord(kf, R.yb, R.yb2, R.dy, R.dy2);
        float z = sample_coord(kf, R.zb, R.zb2, R.dz, R.dz2);
        Cell c = locate(P, z, fmaf(R.x, R.x, y * y));
        n += c.gas ? 1 : 0;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
  if ((threadIdx.x & 31) == 0 && n) atomicAdd(count, n);
}

int launch_count(const MarchParams &P, unsigned long long *count, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return set_error(RT_ECUDA, "count memset: %s", cudaGetErrorString(e));
  if (npix == 0) return RT_OK;
  long long blocks = (npix + 255) / 256;
  count_gas_kernel<<<(unsigned)blocks, 256, 0, stream>>>(P, count);
  e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "count launch: %s", cudaGetErrorString(e));
  return RT_OK;
}

}  // namespace rtb
