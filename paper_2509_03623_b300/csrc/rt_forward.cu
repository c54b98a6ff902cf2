// Forward march kernel.
//
// Mapping: a warp marches R = 32/LPR neighbouring rays at a time (one work unit); the LPR
// lanes of a ray split its channels: lane q holds channels q + LPR j, j < CPL, as CPL/2 pairs,
// pair m = channels (q + 2m LPR, q + (2m+1) LPR), so that pair m of all lanes covers the
// contiguous channel block [2m LPR, (2m+2) LPR). The grid is persistent (one wave) and work
// units are interleaved over its warps; the double-precision ray setups (chord through the
// bounding cylinder) of 32 rays are computed at once, one per lane, and kept in shared memory.
// Samples advance in batches of 2 LPR: in the physics phase lane q evaluates the channel-
// independent physics of samples kb+q and kb+LPR+q of its ray (fields, CO layer, Keplerian
// velocity, line width, LTE source and opacity; two independent evaluations per lane for
// instruction-level parallelism, which the specialised modes issue as two-lane FP32
// instructions, FFMA2 / FMUL2 / FADD2) once and publishes them in shared memory; in the channel
// phase every lane walks the batch's samples in order, evaluating the Doppler-shifted Gaussian
// profile and advancing optical depth, transmittance and intensity front to back (Eq. rt-int
// with Eq. optical_depth; the source is constant over each segment).
//
// Channel window. A sample's optical depth in channel c is kd 2^{-d_c^2}; it is below 2^-40
// (so that a whole ray of skipped contributions changes a transmittance by less than 1e-9)
// once |v_c - v_los| > sqrt(40 + log2 kd) / b. With equally spaced channels each lane turns
// that velocity window of its sample into a range of (fractional) channel indices in the
// physics phase, and a warp vote per channel block decides which blocks any sample of the
// batch reaches; only those blocks are marched (a warp-uniform branch, so the skipped work
// is not issued). Batches without gas reach no block.
//
// Per sample-channel evaluation: 6 FP32 operations, issued as 3 packed two-channel
// instructions (FFMA2/FMUL2/FADD2), and 2 MUFU.EX2. The optical depth is kept negated (so no
// negation is needed before the exponential) and summed per batch, then folded into a
// per-channel base at the end of every batch with Kahan compensation: the fold's rounding
// error is carried into the next batch's sum, so the base is exact to about one rounding of
// the total optical depth however many batches the ray has.
//
// Gas range. Each ray's setup gives the range of samples that can lie inside the gas wedge
// (gas_range); a ray is marched from the first sample of its range, the warp's batches
// running until the longest range of its rays ends. Samples outside the range are exact
// no-ops of the march (no gas), so they are not visited.
#include <mutex>
#include <new>

#include "rt_internal.cuh"

namespace rtb {

constexpr int kWarps = 4;        // warps per block
constexpr float kWinLog2 = 40.0f;  // skipped optical depths are below 2^-40 per sample

// Blocks per SM the register budget is sized for: 5 (at most 102 registers) with 8 channels
// per lane, 6 with 4; 4 (128 registers) for the 3-D grids, whose sample physics holds 16
// node records in flight, and for the specialised modes, whose two-sample physics holds both
// samples' corner quads and intermediates at once (spilled at 96 registers: 0.276 ms against
// 0.255 ms at 128 on the observation-scale disk).
template <int LPR, int CPL, int MODE>
__global__ void __launch_bounds__(kWarps * 32,
                                  (MODE == 2 || MODE == 3 || MODE >= 4) ? 4 : (CPL == 8 ? 5 : 6))
    march_fwd_kernel(const __grid_constant__ MarchParams P, float *__restrict__ cube) {
  constexpr int R = 32 / LPR;  // rays marched together by one warp (one work unit)
  constexpr int G = 32 / R;    // work units whose ray setups are computed together
  constexpr int H = CPL / 2;   // channel pairs per lane = channel blocks
  __shared__ __align__(16) float s_tab[kTabSeg * 4];
  // per sample: {-kd, -kd, S, S} and {b, b, -a, -a} (pairs ready for the packed arithmetic)
  // per ray 2 LPR records plus one float4 of padding, so that the rays of a warp (reading one
  // record each, broadcast to their lanes) fall on different banks
  constexpr int kPhStride = 2 * LPR + 1;
  __shared__ float4 s_ph[kWarps][2][(32 / LPR) * kPhStride];
  __shared__ Ray s_ray[kWarps][32];
  for (int i = threadIdx.x; i < kTabSeg * 4; i += blockDim.x) s_tab[i] = P.tab[i];
  // launched as the prep kernel's programmatic dependent: the ray setups, the counter and the
  // corner quads are complete and visible after this (a no-op in an ordinary launch)
  asm volatile("griddepcontrol.wait;" ::: "memory");
  __syncthreads();

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int q = lane % LPR, rr = lane / LPR;
  const long long npix = (long long)P.nx * P.ny;
  const long long nunits = (npix + R - 1) / R;
  const long long W = (long long)gridDim.x * kWarps;  // warps in the grid
  float4 *ph0 = s_ph[wib][0];
  float4 *ph1 = s_ph[wib][1];

  // velocities of this lane's channel pairs
  float2 vp[H];
#pragma unroll
  for (int m = 0; m < H; m++) {
    const int c0 = q + LPR * (2 * m), c1 = c0 + LPR;
    vp[m] = (MODE >= 4 || P.v_uniform) ? make_float2(fmaf((float)c0, P.dv, P.v0),
                                                     fmaf((float)c1, P.dv, P.v0))
                        : make_float2(P.v[min(c0, RT_MAX_CH - 1)], P.v[min(c1, RT_MAX_CH - 1)]);
  }
  // the window test needs equally spaced channels; otherwise every block is marched
  // the window is tested in channel-index space; without equal spacing every block is marched
  const bool windowed = MODE >= 4 || (P.v_uniform && P.dv != 0.0f && !P.no_window);
  const float idv = windowed ? 1.0f / P.dv : 0.0f;
  const float2 mone = make_float2(-1.0f, -1.0f);
  // work counters (lane 0; only with P.work): samples whose physics found gas, channel
  // evaluations computed (every lane of an active block, LPR samples x 2 channels each)
  unsigned long long wc_phys = 0, wc_eval = 0;

  // One work unit: the R rays of a warp (pixels u R .. u R + R - 1), marched to the cube.
  auto march_unit = [&](long long u, Ray ray) __attribute__((always_inline)) {
      const long long pix = u * R + rr;
      // negated optical depth: batch part and base; transmittance; intensity
      float2 nl[H], nb[H], Tr[H], I[H];
#pragma unroll
      for (int m = 0; m < H; m++) {
        nl[m] = make_float2(0.0f, 0.0f);
        nb[m] = make_float2(0.0f, 0.0f);
        Tr[m] = make_float2(1.0f, 1.0f);
        I[m] = make_float2(0.0f, 0.0f);
      }
      // the rays' gas sample ranges, marched from their first samples (klo) on
      const int nsamp = __reduce_max_sync(0xffffffffu, max(ray.khi - ray.klo + 1, 0));
      for (int kb = 0; kb < nsamp; kb += 2 * LPR) {
        float4 mine, mine2;
        if (MODE >= 4) {
          // the specialised physics of both samples in two-lane arithmetic (same results)
          sample_physics_x2<MODE == 5>(P, s_tab, ray, ray.klo + kb + q, ray.klo + kb + LPR + q,
                                       mine, mine2);
        } else {
          mine = march_physics<MODE>(P, s_tab, ray, ray.klo + kb + q);
          mine2 = march_physics<MODE>(P, s_tab, ray, ray.klo + kb + LPR + q);
        }
        // channel window of each sample (empty without gas): fractional channel indices where
        // kd 2^{-d^2} >= 2^-40; the lane votes with the union of its two samples' windows.
        // Both samples' bounds in two-lane arithmetic; a sample without gas (kd = 0) or whose
        // window is empty (w2 <= 0) gives the empty range.
        float clo = 1e30f, chi = -1e30f;
        if (mine.x > 0.0f || mine2.x > 0.0f) {
          const float2 w2 = __fadd2_rn(bc2(kWinLog2), make_float2(lg2(mine.x), lg2(mine2.x)));
          const float2 ib = make_float2(rcp(mine.z), rcp(mine2.z));
          const float2 hw = __fmul2_rn(make_float2(sqa(w2.x), sqa(w2.y)), ib);
          const float2 vl = __fmul2_rn(make_float2(mine.y, mine2.y), ib);
          const float2 e0 = __fmul2_rn(sub2(sub2(vl, hw), bc2(P.v0)), bc2(idv));
          const float2 e1 = __fmul2_rn(sub2(__fadd2_rn(vl, hw), bc2(P.v0)), bc2(idv));
          if (mine.x > 0.0f && w2.x > 0.0f) {
            clo = fminf(e0.x, e1.x) - 0.01f;
            chi = fmaxf(e0.x, e1.x) + 0.01f;
          }
          if (mine2.x > 0.0f && w2.y > 0.0f) {
            clo = fminf(clo, fminf(e0.y, e1.y) - 0.01f);
            chi = fmaxf(chi, fmaxf(e0.y, e1.y) + 0.01f);
          }
        }
        unsigned act = 0;
        if (windowed) {
#pragma unroll
          for (int m = 0; m < H; m++)
            if (__any_sync(0xffffffffu, chi >= (float)(2 * m * LPR) &&
                                            clo <= (float)((2 * m + 2) * LPR - 1)))
              act |= 1u << m;
        } else if (__any_sync(0xffffffffu, mine.x > 0.0f || mine2.x > 0.0f)) {
          act = (1u << H) - 1;
        }
        if (P.work) {
          const unsigned gl = __ballot_sync(0xffffffffu, mine.x > 0.0f);
          const unsigned gl2 = __ballot_sync(0xffffffffu, mine2.x > 0.0f);
          wc_phys += __popc(gl) + __popc(gl2);
          wc_eval += (unsigned long long)__popc(act) * 128 * LPR;
        }
        if (!act) continue;  // no channel of any ray reached in this batch
        ph0[rr * kPhStride + q] = make_float4(-mine.x, -mine.x, mine.w, mine.w);
        ph1[rr * kPhStride + q] = make_float4(mine.z, mine.z, -mine.y, -mine.y);
        ph0[rr * kPhStride + LPR + q] = make_float4(-mine2.x, -mine2.x, mine2.w, mine2.w);
        ph1[rr * kPhStride + LPR + q] = make_float4(mine2.z, mine2.z, -mine2.y, -mine2.y);
        __syncwarp();
        // one sample of the batch in channel block m: profile, optical depth, transmittance
        // and intensity (samples without gas are exact no-ops)
        auto step = [&](int m, const float4 &p0, const float4 &p1) __attribute__((always_inline)) {
          const float2 nkd = make_float2(p0.x, p0.y), S = make_float2(p0.z, p0.w);
          const float2 b = make_float2(p1.x, p1.y), na = make_float2(p1.z, p1.w);
          const float2 d = __ffma2_rn(vp[m], b, na);  // (v_c - v_los) / alpha (scaled)
          const float2 d2 = __fmul2_rn(d, d);
          const float2 gp = make_float2(ex2(-d2.x), ex2(-d2.y));
          nl[m] = __ffma2_rn(nkd, gp, nl[m]);
          const float2 nt = __fadd2_rn(nb[m], nl[m]);
          const float2 Tn = make_float2(ex2(nt.x), ex2(nt.y));
          const float2 df = __ffma2_rn(Tn, mone, Tr[m]);  // T_k - T_{k+1}
          I[m] = __ffma2_rn(S, df, I[m]);
          Tr[m] = Tn;
        };
        // compensated fold of the batch into the base (Kahan): nl carries the batch sum minus
        // the base's rounding error left by the previous fold
        auto fold = [&](int m) __attribute__((always_inline)) {
          const float2 t = __fadd2_rn(nb[m], nl[m]);
          nl[m] = __ffma2_rn(__ffma2_rn(nb[m], mone, t), mone, nl[m]);
          nb[m] = t;
        };
        // the active blocks (warp-uniform), two adjacent ones in one pass over the batch's
        // samples: each sample's records are read once for both, and the two blocks' chains
        // interleave; every channel sees the same operations in the same order either way
        unsigned rem = act;
#pragma unroll
        for (int m = 0; m < H; m++) {
          if (!(rem & (1u << m))) continue;  // block m outside every window
          if (m + 1 < H && (rem & (2u << m))) {
            rem &= ~(2u << m);
#pragma unroll
            for (int t = 0; t < 2 * LPR; t++) {
              const float4 p0 = ph0[rr * kPhStride + t];
              const float4 p1 = ph1[rr * kPhStride + t];
              step(m, p0, p1);
              step(m + 1 < H ? m + 1 : m, p0, p1);
            }
            fold(m);
            fold(m + 1 < H ? m + 1 : m);
          } else {
#pragma unroll
            for (int t = 0; t < 2 * LPR; t++)
              step(m, ph0[rr * kPhStride + t], ph1[rr * kPhStride + t]);
            fold(m);
          }
        }
        __syncwarp();
      }
      if (pix < npix) {
#pragma unroll
        for (int m = 0; m < H; m++) {
          const int c0 = q + LPR * (2 * m), c1 = c0 + LPR;
          if (c0 < P.nch) cube[(long long)c0 * npix + pix] = fmaf(I[m].x, P.out_scale, P.I0 * Tr[m].x);
          if (c1 < P.nch) cube[(long long)c1 * npix + pix] = fmaf(I[m].y, P.out_scale, P.I0 * Tr[m].y);
        }
      }
  };
  if (P.unit_ctr) {
    // Dynamic: a warp takes one unit at a time from the launch-wide counter, in pixel order,
    // so warps that drew short rays take more units, and the last units handed out are the
    // bottom rows of the image, which cross little gas (a short tail); the ray setups come
    // from the pre-pass.
    for (;;) {
      unsigned uc = 0;
      if (lane == 0) uc = atomicAdd(P.unit_ctr, 1u);
      const long long u = (long long)__shfl_sync(0xffffffffu, uc, 0);
      if (u >= nunits) break;
      const long long pix = u * R + rr;
      march_unit(u, P.rays[pix < npix ? pix : npix - 1]);  // a ray past the end stores nothing
    }
  } else {
    // Static: units u = gw, gw + W, gw + 2W, ... (interleaved over the grid); the setups of G
    // units (32 rays) are computed at once, one ray per lane.
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
        march_unit(u, s_ray[wib][g * R + rr]);
      }
    }
  }
  if (P.work && lane == 0) {
    atomicAdd(P.work, wc_phys);
    atomicAdd(P.work + 1, wc_eval);
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

template <int LPR, int CPL>
static void launch_t(const MarchParams &P, float *cube, cudaStream_t stream, bool pdl) {
  const bool spec = spec_ok(P);
  auto kern = P.sph ? march_fwd_kernel<LPR, CPL, 3>
              : P.box ? march_fwd_kernel<LPR, CPL, 2>
              : P.vphi ? (spec ? march_fwd_kernel<LPR, CPL, 5> : march_fwd_kernel<LPR, CPL, 1>)
                       : (spec ? march_fwd_kernel<LPR, CPL, 4> : march_fwd_kernel<LPR, CPL, 0>);
  long long npix = (long long)P.nx * P.ny;
  long long units = (npix + (32 / LPR) - 1) / (32 / LPR);
  long long need = (units + kWarps - 1) / kWarps;
  long long cap = resident_blocks((const void *)kern, kWarps * 32);
  long long blocks = need < cap ? need : cap;
  // the dynamic march follows its prep kernel as a programmatic dependent launch (pdl)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(kWarps * 32);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kern, P, cube);
}

// Channels per lane (4, or 8 from 32 channels up) and lanes per ray (power of two). Without
// the channel window (the dense march) 4 channels per lane up to 64 channels: more lanes per
// ray and fewer registers per lane (1.02 -> 0.67 ms on 256^2 px x 64 channels x 512 samples),
// where the windowed march needs the narrower 16-channel blocks of 8 lanes x 8 channels.
void lane_layout(int nch, bool dense, int *lpr, int *cpl) {
  int c = (nch >= 32 && !(dense && nch <= 64)) ? 8 : 4;
  int need = (nch + c - 1) / c, l = 1;
  while (l < need) l *= 2;
  *lpr = l;
  *cpl = c;
}

// Corner quads of the node fields (MarchParams::cell, hcell), rebuilt from the caller's
// arrays before every launch that uses them: one thread per cell gathers the four nodes of
// each field that the cell's bilinear interpolation reads.
// Cells first, first + stride, ... of the grid.
__device__ __forceinline__ void pack_cells_from(const float *__restrict__ T,
                                                const float *__restrict__ n,
                                                const float *__restrict__ vt,
                                                const float *__restrict__ hlo,
                                                const float *__restrict__ hhi,
                                                const float *__restrict__ vphi, int nr, int nz,
                                                float4 *__restrict__ cell,
                                                float4 *__restrict__ hcell, long long first,
                                                long long stride) {
  const long long m = (long long)(nr - 1) * (nz - 1);
  for (long long i = first; i < m; i += stride) {
    const int j = (int)(i / (nr - 1)), r = (int)(i - (long long)j * (nr - 1));
    const long long b = (long long)j * nr + r;  // node (r, j); the cell's nodes end at b+nr+1
    const int nq = vphi ? 4 : 3;
    float4 *cq = cell + nq * i;
    cq[0] = make_float4(T[b], T[b + 1], T[b + nr], T[b + nr + 1]);
    cq[1] = make_float4(n[b], n[b + 1], n[b + nr], n[b + nr + 1]);
    cq[2] = make_float4(vt[b], vt[b + 1], vt[b + nr], vt[b + nr + 1]);
    if (vphi) cq[3] = make_float4(vphi[b], vphi[b + 1], vphi[b + nr], vphi[b + nr + 1]);
    if (j == 0) hcell[r] = make_float4(hlo[r], hlo[r + 1], hhi[r], hhi[r + 1]);
  }
}

__global__ void pack_cells_kernel(const float *__restrict__ T, const float *__restrict__ n,
                                  const float *__restrict__ vt, const float *__restrict__ hlo,
                                  const float *__restrict__ hhi,
                                  const float *__restrict__ vphi, int nr, int nz,
                                  float4 *__restrict__ cell, float4 *__restrict__ hcell) {
  pack_cells_from(T, n, vt, hlo, hhi, vphi, nr, nz, cell, hcell,
                  (long long)blockIdx.x * blockDim.x + threadIdx.x,
                  (long long)gridDim.x * blockDim.x);
}

// Everything the dynamic forward march reads besides the caller's arrays, in one launch: the
// ray setups of every pixel (blocks below ray_blocks, one thread per ray), the zeroed work
// counter and, with cell != nullptr, the corner quads (the other blocks). The march is
// launched as its programmatic dependent: its blocks start as this grid's last blocks are
// scheduled, stage their tables, and wait for this grid to finish before they read any of it.
__global__ void march_prep_kernel(const __grid_constant__ MarchParams P, Ray *__restrict__ rays,
                                  unsigned *__restrict__ ctr, unsigned ray_blocks,
                                  float4 *__restrict__ cell, float4 *__restrict__ hcell) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (blockIdx.x < ray_blocks) {
    const long long npix = (long long)P.nx * P.ny;
    const long long pix = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (pix == 0) *ctr = 0u;
    if (pix < npix) rays[pix] = setup_ray(P, (int)(pix % P.nx), (int)(pix / P.nx), true);
  } else if (cell) {
    pack_cells_from(P.T, P.n, P.vt, P.hlo, P.hhi, P.vphi, P.nr, P.nz, cell, hcell,
                    (long long)(blockIdx.x - ray_blocks) * blockDim.x + threadIdx.x,
                    (long long)(gridDim.x - ray_blocks) * blockDim.x);
  }
}

// Samples from which the corner quads pay for their packing pass (a launch and a pass over
// the grid; on the 512 x 256 grid with 33.5 M samples they take 20 % off the forward march).
constexpr long long kCellMinSamples = 1LL << 22;

// Bytes of the corner quads of P, or 0 where the kernels should read the node arrays
// (few samples, or a grid so large that packing it costs more than the loads it saves).
size_t cell_bytes(const MarchParams &P) {
  if (P.nr < 2 || P.nz < 2) return 0;
  const long long samples = (long long)P.nx * P.ny * P.n_samples;
  const long long cells = (long long)(P.nr - 1) * (P.nz - 1);
  if (samples < kCellMinSamples || samples < 8 * cells) return 0;
  return (size_t)((P.vphi ? 4 : 3) * cells + (P.nr - 1)) * sizeof(float4);
}

// Packs the corner quads into buf (cell_bytes(P) bytes, 16-byte aligned) on `stream` and
// points P at them.
int pack_cells(MarchParams &P, void *buf, cudaStream_t stream) {
  const long long cells = (long long)(P.nr - 1) * (P.nz - 1);
  float4 *cell = reinterpret_cast<float4 *>(buf);
  float4 *hcell = cell + (P.vphi ? 4 : 3) * cells;
  const long long nb = (cells + 255) / 256;
  pack_cells_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, stream>>>(
      P.T, P.n, P.vt, P.hlo, P.hhi, P.vphi, P.nr, P.nz, cell, hcell);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(RT_ECUDA, "cell packing: %s", cudaGetErrorString(e));
  P.cell = cell;
  P.hcell = hcell;
  return RT_OK;
}

static int launch_march(const MarchParams &P, float *cube, cudaStream_t stream, bool pdl);

// Kernel timing (rt_kernel_timing): CUDA event pairs recorded around march launches.
namespace {
constexpr int kMaxTimed = 4096;
struct KernelTimer {
  std::mutex mu;
  bool on = false;
  int n = 0;
  cudaEvent_t ev[kMaxTimed][2];
};
KernelTimer &ktimer() {
  static KernelTimer t;
  return t;
}
// A fresh event pair for one launch, or false (timing off, no room, no events).
bool timer_pair(cudaEvent_t *a, cudaEvent_t *b) {
  KernelTimer &t = ktimer();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!t.on || t.n >= kMaxTimed) return false;
  if (cudaEventCreate(a) != cudaSuccess) return false;
  if (cudaEventCreate(b) != cudaSuccess) {
    cudaEventDestroy(*a);
    return false;
  }
  t.ev[t.n][0] = *a;
  t.ev[t.n][1] = *b;
  t.n++;
  return true;
}
void timer_drop_locked(KernelTimer &t) {
  for (int i = 0; i < t.n; i++) {
    cudaEventDestroy(t.ev[i][0]);
    cudaEventDestroy(t.ev[i][1]);
  }
  t.n = 0;
}
}  // namespace

// Forward march. One stream-ordered allocation, freed after the launch, holds the corner
// quads where they pay (packed first), the ray setups of every pixel (a pre-pass) and the
// counter of the march's dynamic work distribution (zeroed first).
int launch_forward(const MarchParams &P, float *cube, cudaStream_t stream) {
  long long npix = (long long)P.nx * P.ny;
  if (npix == 0 || P.nch == 0) return RT_OK;
  const size_t cb = (P.cell ? 0 : cell_bytes(P) + 255) & ~(size_t)255;
  const size_t rb = (ray_buffer_bytes(npix) + 255) & ~(size_t)255;
  char *buf = nullptr;
  cudaError_t e = stream_alloc((void **)&buf, cb + rb + 256, stream);
  if (e != cudaSuccess)
    return set_error(RT_ENOMEM, "forward scratch (%zu bytes): %s", cb + rb + 256,
                     cudaGetErrorString(e));
  MarchParams Q = P;  // passed by value to the kernel: the copy only lives until the launch
  Ray *rays = reinterpret_cast<Ray *>(buf + cb);
  unsigned *ctr = reinterpret_cast<unsigned *>(buf + cb + rb);
  float4 *cell = nullptr, *hcell = nullptr;
  const long long cells = (long long)(P.nr - 1) * (P.nz - 1);
  if (cb) {
    cell = reinterpret_cast<float4 *>(buf);
    hcell = cell + (P.vphi ? 4 : 3) * cells;
  }
  const long long ray_blocks = (npix + 255) / 256;
  long long cell_blocks = cb ? (cells + 255) / 256 : 0;
  if (cell_blocks > 4096) cell_blocks = 4096;
  march_prep_kernel<<<(unsigned)(ray_blocks + cell_blocks), 256, 0, stream>>>(
      P, rays, ctr, (unsigned)ray_blocks, cell, hcell);
  int rc = RT_OK;
  e = cudaGetLastError();
  if (e != cudaSuccess) rc = set_error(RT_ECUDA, "forward prep launch: %s", cudaGetErrorString(e));
  if (rc == RT_OK) {
    if (cb) {
      Q.cell = cell;
      Q.hcell = hcell;
    }
    Q.rays = rays;
    Q.unit_ctr = ctr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    const bool timed = timer_pair(&t0, &t1);  // (then an ordinary launch after the prep)
    if (timed) cudaEventRecord(t0, stream);
    rc = launch_march(Q, cube, stream, !timed);
    if (timed) cudaEventRecord(t1, stream);
  }
  cudaFreeAsync(buf, stream);
  return rc;
}

// The dense comparison march: the same kernel visiting every sample of every ray and every
// channel block, reading the node arrays (no gas range, no channel window, no corner quads).
int launch_forward_dense(const MarchParams &P, float *cube, cudaStream_t stream) {
  if ((long long)P.nx * P.ny == 0 || P.nch == 0) return RT_OK;
  MarchParams Q = P;
  Q.full_range = 1;
  Q.no_window = 1;
  Q.cell = nullptr;
  Q.hcell = nullptr;
  Q.rays = nullptr;  // static work distribution, ray setups in the kernel
  Q.unit_ctr = nullptr;
  return launch_march(Q, cube, stream, false);
}

// pdl: launch as the programmatic dependent of the kernel just before it on the stream.
static int launch_march(const MarchParams &P, float *cube, cudaStream_t stream, bool pdl) {
  int LPR, CPL;
  lane_layout(P.nch, P.no_window, &LPR, &CPL);
  if (CPL == 8) {
    if (LPR == 32) launch_t<32, 8>(P, cube, stream, pdl);
    else if (LPR == 16) launch_t<16, 8>(P, cube, stream, pdl);
    else if (LPR == 8) launch_t<8, 8>(P, cube, stream, pdl);
    else launch_t<4, 8>(P, cube, stream, pdl);
  } else {
    if (LPR == 16) launch_t<16, 4>(P, cube, stream, pdl);
    else if (LPR == 8) launch_t<8, 4>(P, cube, stream, pdl);
    else if (LPR == 4) launch_t<4, 4>(P, cube, stream, pdl);
    else if (LPR == 2) launch_t<2, 4>(P, cube, stream, pdl);
    else launch_t<1, 4>(P, cube, stream, pdl);
  }
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

extern "C" int rt_kernel_timing(int on) {
  rtb::KernelTimer &t = rtb::ktimer();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!on) rtb::timer_drop_locked(t);
  t.on = on != 0;
  return RT_OK;
}

extern "C" int rt_kernel_time(double *total_ms, int *launches) {
  if (!total_ms || !launches) return rtb::set_error(RT_EINVAL, "null argument");
  rtb::KernelTimer &t = rtb::ktimer();
  std::lock_guard<std::mutex> lk(t.mu);
  double sum = 0.0;
  int rc = RT_OK;
  for (int i = 0; i < t.n && rc == RT_OK; i++) {
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(t.ev[i][1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.ev[i][0], t.ev[i][1]);
    if (e != cudaSuccess)
      rc = rtb::set_error(RT_ECUDA, "kernel timing: %s", cudaGetErrorString(e));
    sum += ms;
  }
  *total_ms = rc == RT_OK ? sum : 0.0;
  *launches = rc == RT_OK ? t.n : 0;
  rtb::timer_drop_locked(t);
  return rc;
}
