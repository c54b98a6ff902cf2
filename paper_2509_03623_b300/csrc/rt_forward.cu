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
int resident_blocks(const void *kernel, int threads) {
  struct Entry {
    const void *k;
    int dev, threads, blocks;
  };
  static std::mutex mu;
  static Entry cache[64];
  static int n = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  {
    std::lock_guard<std::mutex> lk(mu);
    for (int i = 0; i < n; i++)
      if (cache[i].k == kernel && cache[i].dev == dev && cache[i].threads == threads)
        return cache[i].blocks;
  }
  int nb = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, 0) != cudaSuccess ||
      nb < 1)
    nb = 1;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
    nsm = 1;
  std::lock_guard<std::mutex> lk(mu);
  if (n < 64) cache[n++] = Entry{kernel, dev, threads, nb * nsm};
  return nb * nsm;
}

template <int LPR, int CPL, bool UNIF>
static void launch_t(const MarchParams &P, float *cube, cudaStream_t stream) {
  auto kern = march_fwd_kernel<LPR, CPL, UNIF>;
  long long npix = (long long)P.nx * P.ny;
  long long units = (npix + (32 / LPR) - 1) / (32 / LPR);
  long long need = (units + kWarps - 1) / kWarps;
  long long cap = resident_blocks((const void *)kern, kWarps * 32);
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
