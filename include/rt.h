/*
 * rt.h -- C interface of the B300 line radiative-transfer library (librt_b300.so).
 *
 * The library renders spectral-line cubes of axisymmetric protoplanetary disks by backward
 * ray tracing, following arXiv 2509.03623, Methods, "Line Radiative Transfer with RadJAX":
 * the integral transfer equation (Eq. rt-int) with the optical depth of Eq. optical_depth,
 * emissivity j_nu = h nu0/(4 pi) n_u A_ul phi and extinction
 * beta_nu = h nu0/(4 pi)(n_l B_lu - n_u B_ul) phi, LTE (Boltzmann) level populations, the
 * Doppler-shifted Gaussian profile phi(nu) with delta_nu = omega.v/c, the line width
 * alpha = sqrt(2kT/m_CO + v_turb^2 c_s^2), and Keplerian rotation (first term of
 * Eq. gas_velocity_pressure).
 *
 * Conventions (the paper leaves them open; fixed here):
 *   - Disk frame: +z along the angular momentum; rotation counter-clockwise about +z.
 *     Observer direction (0, -sin i, cos i); sky basis e_x = (1,0,0), e_y = (0, cos i, sin i).
 *     Image pixel (ix, iy) has centre X = (ix + 1/2 - nx/2) 2 half_fov/nx au (Y likewise);
 *     (x_s, y_s) = (X cos PA + Y sin PA, -X sin PA + Y cos PA). Orthographic rays.
 *   - The ray's chord through the cylinder r <= r_out, |z| <= zr_max r_out is cut into
 *     n_samples equal segments sampled at their midpoints; segment k adds
 *     Tr_k S_k (1 - exp(-dtau_k)) and multiplies the transmittance by exp(-dtau_k).
 *     Rays that miss the cylinder return I0.
 *   - Node grids: r log-spaced (r_log = 1) or linear in [r_in, r_out]; z/r linear in
 *     [0, zr_max]; bilinear interpolation in (grid r coordinate, z/r) of T, n_H2, v_turb;
 *     no gas at r < r_in or |z|/r > zr_max. Surfaces h_lo, h_hi (z/r units) are
 *     interpolated in r.
 *   - CO abundance x_co between the surfaces with logistic edges of width edge_w in z/r
 *     (edge_w = 0: hard steps).
 *   - Channel velocities use the radio convention; line-of-sight velocity positive receding.
 *   - Molecule: rigid rotor J_u -> J_u - 1, E_J = h B J(J+1), g_J = 2J+1, B = B_rot_hz or
 *     nu0/(2 J_u) when B_rot_hz <= 0.
 *   - Output cube [nch][ny][nx] (x fastest), float32, in erg s^-1 cm^-2 Hz^-1 sr^-1
 *     (units = 0) or Jy per pixel (units = 1). I0 is in output units.
 *
 * Memory and ownership: every buffer is owned by the caller and is never freed by the
 * library. Field, surface, cube and gradient pointers are DEVICE pointers on the current
 * device; v_kms is a HOST pointer read during the call. Calls are asynchronous on the given
 * CUDA stream (NULL = the legacy default stream) and return once the work is enqueued.
 *
 * Errors: functions return RT_OK (0) or a negative RT_E* code; rt_last_error() returns a
 * thread-local message for the last failure on the calling thread. Invalid arguments are
 * detected on the host before anything is enqueued.
 */
#ifndef RT_B300_H
#define RT_B300_H

#include <stddef.h>
#include <stdint.h>

/*
 * Scratch memory. Entry points that say they allocate take stream-ordered allocations on
 * the caller's stream from a memory pool the library creates for each device (on first use)
 * and free them on that stream after their kernels; the pool keeps up to 1 GiB of freed
 * memory cached for the next call instead of returning it to the driver.
 */

#ifdef __cplusplus
extern "C" {
#endif

#define RT_OK 0
#define RT_EINVAL (-1)     /* invalid argument (sizes, pointers, non-finite values) */
#define RT_ENOMEM (-2)     /* device or host allocation failed */
#define RT_EBUSY (-3)      /* serving: no admission slot or memory budget now */
#define RT_ETIMEDOUT (-4)  /* a bounded wait ran out */
#define RT_ECUDA (-5)      /* a CUDA runtime call failed */
#define RT_ENOTFOUND (-6)  /* serving: unknown ticket */

#define RT_MAX_CH 256      /* channels per render */

/* (r, z/r) node grid. */
typedef struct {
  int nr, nz;       /* nodes in r and in z/r, each >= 2 */
  int r_log;        /* 1: r nodes log-spaced, 0: linear */
  double r_in_au, r_out_au;
  double zr_max;    /* z/r of the last node row */
} rt_grid;

/* Node fields, DEVICE float32, [nz][nr] row-major (z/r row, r fastest); surfaces [nr]. */
typedef struct {
  const float *T_K;       /* gas temperature [K], > 0 */
  const float *n_h2_cm3;  /* H2 number density [cm^-3] */
  const float *vturb;     /* turbulent velocity [km/s] (Mach number if vturb_mach) */
  const float *h_lo;      /* lower CO surface, z/r */
  const float *h_hi;      /* upper CO surface, z/r */
  double x_co;            /* CO abundance between the surfaces */
  double edge_w;          /* logistic edge width in z/r (0: hard steps) */
  int vturb_mach;         /* 0: alpha^2 = 2kT/m_CO + v_turb^2; 1: + v_turb^2 2kT/m_mol */
  const float *vphi_kms;  /* optional rotation speed v_phi [km/s], [nz][nr] (Eq.
                             gas_velocity_pressure with the pressure term, e.g. from
                             rt_pressure_vphi), interpolated like the other fields and
                             projected as v_los = v_phi (x / r) sin i + v_sys; NULL: the
                             Keplerian term alone, evaluated at each sample. With it the
                             adjoint entry points also return dL/dvphi_kms (rt_grads.dvphi,
                             required then). */
} rt_fields;

/* Viewing geometry and kinematics. */
typedef struct {
  double incl_deg, pa_deg;
  double dist_pc;       /* used for Jy per pixel */
  double mstar_msun;    /* Keplerian rotation */
  double vsys_kms;      /* systemic velocity added to omega.v */
} rt_geom;

/* Image and spectral sampling. */
typedef struct {
  int nx, ny;           /* pixels (0 allowed: nothing to do; nx*ny <= 2^31) */
  double half_fov_au;   /* <= 0: 1.1 r_out */
  int nch;              /* 0..RT_MAX_CH */
  const float *v_kms;   /* HOST [nch] channel velocities */
  int n_samples;        /* samples per ray, 1 .. 2^20 */
  double I0;            /* background intensity, output units */
  int units;            /* 0: erg s^-1 cm^-2 Hz^-1 sr^-1, 1: Jy per pixel */
} rt_view;

/* Line constants (rigid rotor J_u -> J_u - 1). */
typedef struct {
  double nu0_hz;        /* rest frequency */
  double A_ul;          /* Einstein A [s^-1] */
  double B_rot_hz;      /* rotational constant; <= 0: nu0 / (2 J_u) */
  double m_co_amu;      /* emitting molecule mass (thermal width) */
  double m_mol_amu;     /* mean molecular mass (Mach-mode sound speed) */
  int J_u;              /* upper level, >= 1 */
} rt_line;

/*
 * rt_render -- forward march (Eq. rt-int / Eq. optical_depth, front to back).
 * Writes the cube [nch][ny][nx] float32 to `cube` (DEVICE, caller-allocated,
 * nch*ny*nx floats). Arithmetic is FP32 (optical depth summed in blocks of samples). With
 * equally spaced channels each sample's optical depth is evaluated only in the channel blocks
 * where kd 2^{-d^2} can reach 2^-40 (d the profile argument; below that a whole ray of
 * contributions moves a transmittance by less than 1e-9, far below FP32 relevance); the
 * result is the dense march's. No device memory is allocated. Returns RT_OK, RT_EINVAL or
 * RT_ECUDA (launch failure).
 */
int rt_render(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
              const rt_view *view, const rt_line *line, float *cube, void *stream);

/*
 * rt_count_gas_samples -- work count of a render: the number of (ray, sample) pairs whose
 * sample lies inside the gas grid (r >= r_in, |z|/r <= zr_max) on rays that hit the bounding
 * cylinder, i.e. the samples the march evaluates (sampling rule as in rt_render).
 * `count` is a DEVICE pointer to one unsigned 64-bit integer, overwritten (stream-ordered).
 * Field arrays are not read. Returns RT_OK, RT_EINVAL or RT_ECUDA.
 */
int rt_count_gas_samples(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                         const rt_view *view, const rt_line *line, unsigned long long *count,
                         void *stream);

/* Gradient outputs of rt_render_adjoint: DEVICE float64 arrays, overwritten by the call. */
typedef struct {
  double *dT;       /* [nz][nr] dL/dT_K */
  double *dn;       /* [nz][nr] dL/dn_h2 */
  double *dvt;      /* [nz][nr] dL/dvturb */
  double *dh_lo;    /* [nr] dL/dh_lo */
  double *dh_hi;    /* [nr] dL/dh_hi */
  double *loss;     /* 1 value: sum over voxels of (cube - target)^2 when a target is given;
                       may be NULL */
  double *dvphi;    /* [nz][nr] dL/dvphi_kms (per km/s): required when the fields carry a
                       rotation field (rt_fields.vphi_kms), unused otherwise */
} rt_grads;

/*
 * rt_render_plain -- the plain FP32 march that the forward's throughput is compared against:
 * the same transfer, physics and sampling as rt_render (Keplerian rotation only), computed
 * the straightforward way -- one thread per (pixel, channel) evaluating every sample's
 * physics itself, fields from the node arrays, accurate FP32 library functions, no channel
 * window, no corner quads, plain FP32 sums. Arguments and output as rt_render; its cube
 * agrees with rt_render's within the forward parity criterion. A measurement baseline, not a
 * production path.
 * Returns RT_OK, RT_EINVAL (as rt_render, or a rotation field) or RT_ECUDA.
 */
int rt_render_plain(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                    const rt_view *view, const rt_line *line, float *cube, void *stream);

/*
 * rt_render_dense -- the dense FP32 march the forward is also compared against: rt_render's
 * kernel (one warp per group of rays, the channel-independent physics of each sample computed
 * once and shared by its channels, packed two-channel FP32 arithmetic) with its two work
 * skips removed -- every sample of every ray's chord is visited (no gas sample range) and
 * every channel of every sample is evaluated (no channel window) -- and the fields read from
 * the node arrays (no corner quads). Same transfer (Methods, Eq. rt-int, Eq. optical_depth)
 * and arguments as rt_render; its cube agrees with rt_render's to FP32 rounding. A
 * measurement baseline, not a production path. Returns RT_OK, RT_EINVAL or RT_ECUDA.
 */
int rt_render_dense(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                    const rt_view *view, const rt_line *line, float *cube, void *stream);

/*
 * rt_render_launch_count -- number of kernel launches rt_render makes for this problem
 * (written to *count, HOST): 0 for an empty image or channel list, 2 when it packs the corner
 * quads first (from 4M samples, see rt_render), else 1. Nothing is launched. Returns RT_OK or
 * RT_EINVAL.
 */
int rt_render_launch_count(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                           const rt_view *view, const rt_line *line, int *count);

/*
 * rt_render_work -- rt_render that also counts its work into work (DEVICE, 2 x uint64,
 * overwritten): work[0] = samples with gas whose channel-independent physics was evaluated,
 * work[1] = sample-channel evaluations computed (after the channel window). For roofline
 * accounting; the cube is identical to rt_render's. Returns as rt_render.
 */
int rt_render_work(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                   const rt_view *view, const rt_line *line, float *cube,
                   unsigned long long *work, void *stream);

/*
 * rt_render_adjoint -- forward march plus its reverse-mode gradient (the paper obtains the
 * same gradient by automatic differentiation of the renderer, Methods, "Line Radiative
 * Transfer with RadJAX" and Fig. 2; here it is a hand-written fused adjoint).
 * Seed: exactly one of
 *   dL_dcube  DEVICE [nch][ny][nx] float32, the gradient of a scalar loss w.r.t. the cube, or
 *   target    DEVICE [nch][ny][nx] float32; the loss is L = sum (cube - target)^2 and
 *             dL/dcube = 2 (cube - target) is formed in the kernel (the loss value goes to
 *             grads->loss if non-NULL).
 * cube_out (DEVICE, may be NULL) receives the rendered cube (same values as rt_render up to
 * FP32 rounding). Gradients w.r.t. every node of T, n_H2, v_turb and both surfaces
 * overwrite the FP64 arrays; with a rotation field (fields->vphi_kms) so does its gradient
 * (grads->dvphi, required then), through v_los = v_phi sin i x / r + v_sys. The call
 * allocates and frees one device scratch buffer on `stream` (stream-ordered) holding, per warp
 * of the persistent grid, the optical depths the forward pass keeps at every batch boundary
 * (8 bytes per lane for each channel pair a batch advanced, and a one-byte pair mask per
 * batch; the reverse pass walks the batches back to front from them, with each sample's
 * physics and local derivatives in shared memory), and up to 32 replicated FP32
 * copies of the node gradients (at most 16 MiB, {dT, dn, dvt, dvphi} interleaved per node) plus up
 * to 128 of the surface gradients: each block of the kernel reduces into one copy, and the
 * copies are summed in FP64, in a fixed order, into the outputs at the end. Atomics on one
 * address are applied one after another, and without the copies the surface entries, which
 * every sample at a given radius updates, serialize the kernel. Each copy entry sums a few
 * hundred contributions in FP32 in an order the device does not fix, so repeated calls agree
 * to about 1e-7 of the largest gradient, not bit for bit (the cube is reproducible bit for
 * bit, the loss to FP64 rounding). Where no copies are used, contributions go straight into the outputs as
 * FP64 atomics.
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_render_adjoint(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                      const rt_view *view, const rt_line *line, const float *dL_dcube,
                      const float *target, float *cube_out, const rt_grads *grads, void *stream);

/*
 * rt_render_adjoint_work -- rt_render_adjoint (same arguments, results and errors) that also
 * counts the work its kernel does (measurement support; no counterpart in the paper).
 * `work` is a DEVICE pointer to four unsigned 64-bit counters, overwritten (stream-ordered):
 *   [0] samples whose physics found gas (opacity > 0) in the forward pass,
 *   [1] sample-channel evaluations computed in the forward pass (after the channel window),
 *   [2] 0 (a recompute pass of an earlier design; the counter is kept for the layout),
 *   [3] evaluations computed in the reverse pass.
 */
int rt_render_adjoint_work(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                           const rt_view *view, const rt_line *line, const float *dL_dcube,
                           const float *target, float *cube_out, const rt_grads *grads,
                           unsigned long long *work, void *stream);

/*
 * rt_render_adjoint_noalloc -- rt_render_adjoint for callers that cannot allocate device
 * memory. The paper has no counterpart: this is a deployment variant of the same fused
 * adjoint. Some callers cannot call cudaMalloc or cudaMallocAsync, or have it called for
 * them: for example an application whose memory manager has already reserved the device's
 * memory, or a service that runs under a fixed device-memory budget and allows no allocator
 * traffic once it is running. This entry point performs no device or host allocation: its
 * scratch (checkpoints, and replicated gradient accumulators where room is left) is one
 * fixed 32 MiB array in the library's device memory, which every GPU that loads the library
 * holds until the process exits.
 * Arguments, seeds, outputs and results are those of rt_render_adjoint. In addition:
 *   - The first call on a device looks up the array's device address (with that device
 *     current) and caches it with the ID of the current CUDA context; make that first call
 *     before any stream capture. A call in another context of that device (after
 *     cudaDeviceReset, for example, which unloads the library's device code) looks the
 *     address up again.
 *   - Every call on a device shares the same array. Each call clears what it needs (the
 *     checkpoints are written before they are read, the gradient copies are zeroed on
 *     `stream`), but calls whose kernels overlap on the GPU (different streams, or different
 *     host threads) race on the array: serialize them.
 *   - Checkpoints (the optical depths the forward pass keeps at every batch boundary) get
 *     at most 24 MiB of the array. When that cannot hold checkpoints for a full grid, fewer
 *     blocks are launched; where fewer gradient copies fit (or none: then the kernel adds
 *     straight into the FP64 output arrays), the sums run in another order. Same results up
 *     to that rounding (about 1e-7 of the largest gradient), lower throughput. A problem
 *     whose single block needs more than 24 MiB of checkpoints is rejected with RT_EINVAL and
 *     a message naming the limit: above 24,526 samples per ray with up to 8 channels, 24,548
 *     with 32, 49,052 with 9 to 16, 49,096 with 33 to 64, 98,104 with 17 to 31, 196,400 with
 *     65 to 128 and 392,800 with 129 to 256.
 * Returns RT_OK, RT_EINVAL or RT_ECUDA.
 */
int rt_render_adjoint_noalloc(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                              const rt_view *view, const rt_line *line, const float *dL_dcube,
                              const float *target, float *cube_out, const rt_grads *grads,
                              void *stream);

/*
 * rt_field_chain -- physics-constrained field chain: from a temperature grid to the H2
 * density, the H2 column and the CO layer that the march reads (Methods, "Parametric Disk
 * Modeling": Eq. gas_density_temp, the surface-density profile Sigma(r), Eq. column_density
 * and Eq. co_layer; "Neural Temperature Recovery" derives these fields from the temperature).
 * Per radius node r_i, on the node heights z_j = w_j r_i (w_j = j zr_max / (nz - 1)):
 *   d ln rho / dz = -G M z m_mol / ((r^2 + z^2)^{3/2} k T) - d ln T / dz, integrated upward
 *     from the midplane by the trapezoid rule on the nodes (the ln T term exactly);
 *   rho scaled so that 2 int_0^{z_max} rho dz (trapezoid, mirror symmetry) = Sigma(r),
 *     Sigma(r) = sigma0 (r / r_c)^-gamma exp(-(r / r_c)^{2 - gamma});
 *   n_h2 = rho / m_mol (line->m_mol_amu);  N_h2(z_j) = int_{z_j}^{z_max} n_h2 dz (trapezoid);
 *   the CO layer {T > T_freeze, 0.706 N_h2 > N_dissoc} as two surfaces in z/r:
 *     h_lo = lowest w with T > T_freeze (T linear between nodes; 0 if the midplane node is
 *            warmer, zr_max if no node is),
 *     h_hi = highest w with 0.706 N_h2 > N_dissoc (N_h2 linear between nodes; 0 if none).
 * grid: nodes and r spacing as for the render; geom->mstar_msun: M (>= 0).
 * T: DEVICE [nz][nr] float32, > 0. Outputs (DEVICE, caller-allocated, overwritten):
 *   n_h2 [nz][nr] float32 [cm^-3], N_h2 [nz][nr] float32 [cm^-2] (may be NULL),
 *   h_lo, h_hi [nr] float32 (z/r; usable as rt_fields surfaces).
 * FP32 arithmetic; one warp per radius column.
 * Returns RT_OK, RT_EINVAL (null pointer, grid with fewer than 2 nodes per axis, non-finite
 * or out-of-range parameter) or RT_ECUDA.
 */
typedef struct {
  double sigma0_gcm2;   /* Sigma0 [g cm^-2], >= 0 */
  double r_c_au;        /* characteristic radius [au], > 0 */
  double gamma;         /* surface-density power-law index, < 2 */
  double T_freeze_K;    /* freeze-out temperature [K] */
  double N_dissoc_cm2;  /* photodissociation threshold on 0.706 N_H2 [cm^-2], >= 0 */
} rt_chain;

int rt_field_chain(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                   const rt_chain *chain, const float *T_K, float *n_h2, float *N_h2,
                   float *h_lo, float *h_hi, void *stream);

/*
 * rt_field_chain_adjoint -- reverse mode of rt_field_chain for a scalar loss L (the paper
 * trains its neural temperature through these fields, "Neural Temperature Recovery"): from
 *   g_n  = dL/dn_h2, DEVICE [nz][nr] float64 (e.g. rt_render_adjoint's grads->dn),
 *   g_lo = dL/dh_lo, g_hi = dL/dh_hi, DEVICE [nr] float64 (grads->dh_lo, grads->dh_hi),
 * any of them NULL for zero, writes g_T = dL/dT_K through this chain, DEVICE [nz][nr] float64,
 * caller-allocated, overwritten: through the hydrostatic integration and its normalisation
 * (n_h2), the column N_h2 (h_hi) and the freeze-out crossing (h_lo). A surface depends on the
 * two nodes of the cell where its threshold is crossed, through the linear interpolation in
 * that cell (which cell is piecewise constant in T); a surface pinned at 0 or zr_max has zero
 * derivative. The gradient of a render of the chain's fields with respect to T is g_T plus
 * the render adjoint's own grads->dT. Arguments grid, geom, line, chain and T_K as for
 * rt_field_chain. One warp per radius column, FP32 arithmetic with the running sums as warp
 * scans (the forward quantities are recomputed); a stream-ordered scratch of 8 bytes per node
 * from the library's pool.
 * Returns RT_OK, RT_EINVAL (as rt_field_chain, or a null g_T), RT_ENOMEM or RT_ECUDA.
 */
int rt_field_chain_adjoint(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                           const rt_chain *chain, const float *T_K, const double *g_n,
                           const double *g_lo, const double *g_hi, double *g_T, void *stream);

/*
 * rt_render3d -- forward march through a general 3-D Cartesian grid (the RadJAX setting
 * beyond the axisymmetric disk: Methods, "Line Radiative Transfer with RadJAX", and the
 * 3-D grids of its runtime benchmark): the same transfer (Eq. rt-int / Eq. optical_depth),
 * LTE source and opacity, line width and Doppler-shifted Gaussian profile as rt_render, with
 * the fields interpolated trilinearly on the nodes and the line-of-sight velocity taken from
 * a gas velocity field: v_los = omega . v + v_sys (omega = (0, sin i, -cos i)).
 * Rays are the pixels of rt_view seen at geom's inclination and position angle; each ray's
 * chord through the box [x0, x1] x [y0, y1] x [z0, z1] (disk frame, au) is split into
 * n_samples equal segments with midpoint samples; rays missing the box return I0. Default
 * half field of view: 1.1 times the largest |extent|. geom->mstar_msun is not used.
 * grid3: nodes uniformly spaced, nx, ny, nz >= 2 each, nx*ny*nz <= 2^28.
 * fields3: DEVICE float32 [nz][ny][nx] (x fastest): T_K (> 0), n_h2_cm3, vturb (km/s, or the
 *   Mach number with vturb_mach), x_co (CO abundance per H2), vx, vy, vz (km/s).
 * cube: DEVICE [nch][ny][nx] float32, caller-allocated, overwritten.
 * The call packs the node fields into two float4 records per node (a stream-ordered
 * allocation of 32 bytes per node, freed after the launch). Its reverse mode is
 * rt_render3d_adjoint (below).
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
typedef struct {
  int nx, ny, nz;
  double x0_au, x1_au, y0_au, y1_au, z0_au, z1_au;
} rt_grid3;

typedef struct {
  const float *T_K, *n_h2_cm3, *vturb, *x_co;
  const float *vx_kms, *vy_kms, *vz_kms;
  int vturb_mach;
} rt_fields3;

int rt_render3d(const rt_grid3 *grid3, const rt_fields3 *fields3, const rt_geom *geom,
                const rt_view *view, const rt_line *line, float *cube, void *stream);

/*
 * rt_pack_nodes3 -- the node records the 3-D renders read, packed once so that several
 * renders of the same fields (other views, channel sets, image sizes: the sweeps of the paper's
 * runtime benchmark) skip the packing each rt_render3d / rt_render_sph call does. No
 * counterpart in the paper (a re-layout of its fields; the renders are those of Eq. rt-int).
 * fields3: DEVICE float32 node fields as rt_render3d takes them; for a spherical grid pass
 *   v_r, v_theta, v_phi as vx_kms, vy_kms, vz_kms (vturb_mach is not read here).
 * nodes: number of nodes (nx ny nz, or nr nth nph), 1 .. 2^28.
 * records: DEVICE, 16-byte aligned, 32 bytes x nodes, caller-allocated and owned, overwritten:
 *   nodes float4 {T_K, n_h2_cm3, vturb, x_co} followed by nodes float4 {v0, v1, v2, 0}, in the
 *   fields' node order. Stream-ordered on `stream`; the records depend on nothing else.
 * Returns RT_OK, RT_EINVAL or RT_ECUDA.
 */
int rt_pack_nodes3(const rt_fields3 *fields3, long long nodes, void *records, void *stream);

/*
 * rt_render3d_packed (and rt_render_sph_packed, declared after the spherical grid's types) --
 * rt_render3d / rt_render_sph from node records
 * packed by rt_pack_nodes3 for the same grid (same results bit for bit; no packing and no
 * node-record allocation in the call). vturb_mach as rt_fields3.vturb_mach /
 * rt_fields_sph.vturb_mach; the other arguments as the unpacked renders.
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_render3d_packed(const rt_grid3 *grid3, const void *records, int vturb_mach,
                       const rt_geom *geom, const rt_view *view, const rt_line *line,
                       float *cube, void *stream);

/* Gradient outputs of rt_render3d_adjoint: DEVICE float64 arrays [nz][ny][nx] (x fastest,
   like the fields of rt_fields3), overwritten by the call. */
typedef struct {
  double *dT;      /* dL/dT_K */
  double *dn_h2;   /* dL/dn_h2_cm3 */
  double *dvturb;  /* dL/dvturb (per the vturb input's unit) */
  double *dx_co;   /* dL/dx_co */
  double *dvx;     /* dL/dvx_kms: zero (v_los = omega . v has no x component) */
  double *dvy;     /* dL/dvy_kms (per km/s) */
  double *dvz;     /* dL/dvz_kms (per km/s) */
  double *loss;    /* 1 value: sum over voxels of (cube - target)^2 when a target is given;
                      may be NULL */
} rt_grads3;

/*
 * rt_render3d_adjoint -- fused reverse mode of rt_render3d: the gradient of a scalar loss L
 * with respect to every node of the seven fields of a 3-D Cartesian grid (the reverse march
 * of Eq. rt-int / Eq. optical_depth, as rt_render_adjoint, differentiated through the
 * trilinear interpolation; RadJAX obtains these gradients by automatic differentiation:
 * Methods, "Line Radiative Transfer with RadJAX"). Inputs as rt_render3d. Give exactly one of
 *   dL_dcube  DEVICE [nch][ny][nx] float32: dL/dcube of the caller's loss, or
 *   target    DEVICE [nch][ny][nx] float32: L = sum (cube - target)^2, formed in the kernel.
 * cube_out: DEVICE [nch][ny][nx] float32 receiving the rendered cube (may be NULL).
 * grads: outputs (rt_grads3), all seven arrays required; loss optional.
 * The call allocates (stream-ordered, freed after the launch) the node records (32 bytes per
 * node), one FP32 gradient copy (24 bytes per node) and the per-warp optical depths the
 * forward pass keeps at every batch boundary; node gradients are FP32 sums per node, written
 * out in FP64.
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_render3d_adjoint(const rt_grid3 *grid3, const rt_fields3 *fields3, const rt_geom *geom,
                        const rt_view *view, const rt_line *line, const float *dL_dcube,
                        const float *target, float *cube_out, const rt_grads3 *grads,
                        void *stream);

/*
 * rt_render_sph -- forward march through a 3-D spherical grid centred on the star. RadJAX
 * runs on regularly or log-spaced Cartesian or spherical grids (Methods, "Line Radiative
 * Transfer with RadJAX"), and its runtime benchmark renders a hydrodynamic simulation held
 * on a 512 x 96 x 256 spherical grid. Same transfer (Eq. rt-int / Eq. optical_depth), LTE
 * source and opacity, line width and Doppler-shifted Gaussian profile as rt_render3d, with
 * the fields interpolated trilinearly in (radial index, theta, phi), periodic in phi, and
 *   v_los = omega . v + v_sys,  v = v_r r^ + v_theta theta^ + v_phi phi^,
 * omega = (0, sin i, -cos i), theta the colatitude from the disk's +z axis, phi = atan2(y, x)
 * in [0, 2 pi) in the disk frame (on the axis theta^ and phi^ are taken as 0).
 * Rays are the pixels of rt_view seen at geom's inclination and position angle; each ray's
 * chord through the sphere r <= r_out is split into n_samples equal segments with midpoint
 * samples; samples with r < r_in or theta outside [th0, th1] carry no gas; rays missing the
 * sphere return I0. Default half field of view: 1.1 r_out. geom->mstar_msun is not used.
 * grid: nr >= 2 radial nodes, log-spaced (r_log = 1, r_in > 0) or linear (r_log = 0,
 *   r_in >= 0) over [r_in, r_out] au; nth >= 2 colatitude nodes linear over [th0, th1]
 *   (0 <= th0 < th1 <= pi, radians); nph >= 1 azimuth nodes at phi_k = 2 pi k / nph;
 *   nr*nth*nph <= 2^28.
 * fields: DEVICE float32 [nph][nth][nr] (r fastest): T_K (> 0), n_h2_cm3, vturb (km/s, or the
 *   Mach number with vturb_mach), x_co (CO abundance per H2), and the velocity components
 *   vr_kms, vth_kms, vph_kms (km/s).
 * cube: DEVICE [nch][ny][nx] float32, caller-allocated, overwritten.
 * The call packs the node fields into two float4 records per node (a stream-ordered
 * allocation of 32 bytes per node, freed after the launch). Its reverse mode is
 * rt_render_sph_adjoint (below).
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
typedef struct {
  int nr, nth, nph, r_log;
  double r_in_au, r_out_au, th0_rad, th1_rad;
} rt_grid_sph;

typedef struct {
  const float *T_K, *n_h2_cm3, *vturb, *x_co;
  const float *vr_kms, *vth_kms, *vph_kms;
  int vturb_mach;
} rt_fields_sph;

int rt_render_sph(const rt_grid_sph *grid, const rt_fields_sph *fields, const rt_geom *geom,
                  const rt_view *view, const rt_line *line, float *cube, void *stream);

/*
 * rt_render_sph_adjoint -- fused reverse mode of rt_render_sph: the gradient of a scalar loss
 * with respect to every node of the seven fields of the spherical grid, as
 * rt_render3d_adjoint does for the Cartesian grid (the reverse march of Eq. rt-int /
 * Eq. optical_depth through the trilinear interpolation in (radial index, theta, phi),
 * periodic in phi, and through v_los = omega . (v_r r^ + v_theta theta^ + v_phi phi^)).
 * Inputs as rt_render_sph; dL_dcube / target / cube_out as rt_render3d_adjoint.
 * grads (rt_grads3): all seven arrays required, each [nph][nth][nr] like the fields; dvx, dvy
 * and dvz receive dL/dvr_kms, dL/dvth_kms and dL/dvph_kms (per km/s); loss optional.
 * The call allocates (stream-ordered, freed after the launch) the node records (32 bytes per
 * node), one FP32 gradient copy (32 bytes per node) and the per-warp optical depths kept at
 * every batch boundary.
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_render_sph_adjoint(const rt_grid_sph *grid, const rt_fields_sph *fields,
                          const rt_geom *geom, const rt_view *view, const rt_line *line,
                          const float *dL_dcube, const float *target, float *cube_out,
                          const rt_grads3 *grads, void *stream);

/* rt_render_sph from node records packed by rt_pack_nodes3 (see rt_render3d_packed). */
int rt_render_sph_packed(const rt_grid_sph *grid, const void *records, int vturb_mach,
                         const rt_geom *geom, const rt_view *view, const rt_line *line,
                         float *cube, void *stream);

/*
 * rt_render3d_adjoint_packed / rt_render_sph_adjoint_packed -- rt_render3d_adjoint /
 * rt_render_sph_adjoint from node records packed by rt_pack_nodes3 for the same grid (no
 * packing and no node-record allocation in the call; the same gradients up to the order of
 * the FP32 reductions). vturb_mach as the fields' flag; the other arguments as the unpacked
 * adjoints. Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_render3d_adjoint_packed(const rt_grid3 *grid3, const void *records, int vturb_mach,
                               const rt_geom *geom, const rt_view *view, const rt_line *line,
                               const float *dL_dcube, const float *target, float *cube_out,
                               const rt_grads3 *grads, void *stream);
int rt_render_sph_adjoint_packed(const rt_grid_sph *grid, const void *records, int vturb_mach,
                                 const rt_geom *geom, const rt_view *view, const rt_line *line,
                                 const float *dL_dcube, const float *target, float *cube_out,
                                 const rt_grads3 *grads, void *stream);

/*
 * rt_pressure_vphi -- pressure-corrected rotation on the nodes (Methods, "Parametric Disk
 * Modeling", Eq. gas_velocity_pressure; "Neural Temperature Recovery" derives v_phi from
 * the density and temperature this way):
 *   v_phi^2 = G M r^2 / (r^2 + z^2)^{3/2} + (r / rho) dP/dr |_z,  P = n_H2 k T,
 *   rho = m_mol n_H2 (line->m_mol_amu), M = geom->mstar_msun,
 * with dP/dr at constant z from the grid coordinates (u = ln r on a log grid, r on a linear
 * one; w = z/r): dP/dr |_z = (du/dr) dP/du |_w - (w / r) dP/dw |_u, each a second-order
 * central difference over the nodes (second-order one-sided at the first and last node,
 * first order on a two-node axis). Where v_phi^2 < 0 (pressure support beyond gravity) the
 * result is 0; a node with n_H2 = 0 keeps the Keplerian term.
 * n_h2, T_K: DEVICE [nz][nr] float32; vphi_kms: DEVICE [nz][nr] float32, overwritten (km/s,
 * usable as rt_fields.vphi_kms). FP32, one thread per node.
 * Returns RT_OK, RT_EINVAL (null pointer, grid with fewer than 2 nodes per axis, invalid
 * extent, mass or molecular mass) or RT_ECUDA.
 */
int rt_pressure_vphi(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                     const float *n_h2, const float *T_K, float *vphi_kms, void *stream);

/*
 * rt_pressure_vphi_adjoint -- reverse mode of rt_pressure_vphi for a scalar loss L: from
 * g_vphi = dL/dvphi_kms (DEVICE [nz][nr] float64, e.g. rt_render_adjoint's grads->dvphi)
 * writes g_n = dL/dn_h2 and g_T = dL/dT_K (DEVICE [nz][nr] float64, caller-allocated,
 * overwritten) through the pressure term: the 1/rho factor and the difference stencils
 * transposed. Nodes clamped to v_phi = 0 and nodes with n_H2 = 0 (Keplerian term only)
 * contribute nothing. Arguments grid, geom, line, n_h2 and T_K as for rt_pressure_vphi.
 * FP32 per node, the stencil scatter with FP64 atomics into a stream-ordered scratch of 8 bytes
 * per node.
 * Returns RT_OK, RT_EINVAL (as rt_pressure_vphi), RT_ENOMEM or RT_ECUDA.
 */
int rt_pressure_vphi_adjoint(const rt_grid *grid, const rt_geom *geom, const rt_line *line,
                             const float *n_h2, const float *T_K, const double *g_vphi,
                             double *g_n, double *g_T, void *stream);

/*
 * rt_surface_powerlaw_grad -- chain rule from surface-node gradients to the parameters of a
 * power-law surface h(r) = c (r / 100 au)^p m(r) (m: any fixed modulation):
 *   out[0] = dL/dc = sum_i dL/dh_i h_i / c,   out[1] = dL/dp = sum_i dL/dh_i h_i ln(r_i/100 au),
 * with r_i the grid's r nodes. dh: DEVICE [nr] float64; h: DEVICE [nr] float32 (the surface
 * values used in the render); out: DEVICE 2 float64 (overwritten). Returns RT_OK, RT_EINVAL or
 * RT_ECUDA.
 */
int rt_surface_powerlaw_grad(const rt_grid *grid, const double *dh, const float *h, double c,
                             double *out, void *stream);

/* ------------------------------------------------------------------------------------- */
/* Neural field (Methods, "Neural Temperature Recovery": T(r,|z|) = MLP_w(gamma(r,|z|)))    */
/* ------------------------------------------------------------------------------------- */
/* Network: inputs x = (rhat, zhat), the normalised grid coordinates of a sample (rhat =
 * fractional r node index / (nr-1), zhat = (|z|/r) / zr_max); features
 * [sin 2 pi B x, cos 2 pi B x] for n_freq directions B; Linear layers with SiLU after every
 * hidden layer. Supported shape: n_freq = 32, hidden = 4 layers of width 128, n_out = 4.
 * Outputs o modulate the grid fields at each sample: T <- T e^{o0}, n_H2 <- n_H2 e^{o1},
 * h_lo <- h_lo + h_scale o2, h_hi <- h_hi + h_scale o3. */
#define RT_MLP_F16 0   /* tensor-core operands in FP16 (10-bit mantissa) */
#define RT_MLP_BF16 1  /* tensor-core operands in BF16 (7-bit mantissa) */

typedef struct {
  int n_freq, width, hidden, n_out;
  const float *B;     /* DEVICE [n_freq][2] */
  const float *W[5];  /* DEVICE float32 master weights per Linear layer, [out][in] */
  const float *b[5];  /* DEVICE float32 biases [out] */
  double h_scale;     /* surface offset scale */
  int precision;      /* RT_MLP_F16 or RT_MLP_BF16: 16-bit format of the weights, features
                         and hidden activations fed to the tensor cores (FP32 accumulation) */
} rt_mlp;

/*
 * rt_mlp_eval -- network outputs for n inputs xy [n][2] (DEVICE float32) into out [n][4]
 * (DEVICE float32). Runs on the tensor cores (tcgen05.mma; weights, features and hidden
 * activations rounded to the 16-bit format of mlp->precision, FP32 accumulation in tensor
 * memory, SiLU from the hardware tanh).
 * Returns RT_OK, RT_EINVAL or RT_ECUDA.
 */
int rt_mlp_eval(const rt_mlp *mlp, const float *xy, float *out, long long n, void *stream);

/*
 * rt_render_mlp -- forward render with the neural field: the network is evaluated on the
 * tensor cores (as rt_mlp_eval) at every (pixel, sample) inside the gas grid, its outputs
 * modulate the interpolated grid fields there (see rt_mlp), and the march proceeds as in
 * rt_render. The per-sample outputs go through a device buffer of 16 n_pix n_samples bytes
 * that the call allocates and frees on `stream` (stream-ordered). Returns RT_OK, RT_EINVAL,
 * RT_ENOMEM or RT_ECUDA.
 */
int rt_render_mlp(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                  const rt_view *view, const rt_line *line, const rt_mlp *mlp, float *cube,
                  void *stream);

/*
 * rt_sample_coords -- network inputs (rhat, zhat) of every (pixel, sample) as
 * xy [n_pix][n_samples][2] float32 (DEVICE), (-1, -1) where the sample has no gas. With
 * rt_render_modulated it lets any other evaluation of the network (e.g. in FP32) drive the
 * same march. Field arrays are not read. Returns RT_OK, RT_EINVAL or RT_ECUDA.
 */
int rt_sample_coords(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                     const rt_view *view, const rt_line *line, float *xy, void *stream);

/*
 * rt_render_modulated -- rt_render with per-sample network outputs mod [n_pix][n_samples][4]
 * float32 (DEVICE) applied as in rt_render_mlp with surface offset scale h_scale.
 */
int rt_render_modulated(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                        const rt_view *view, const rt_line *line, const float *mod,
                        double h_scale, float *cube, void *stream);

/* Gradients of a scalar loss with respect to the network parameters (DEVICE float64, same
 * shapes as rt_mlp.W and rt_mlp.b; overwritten by the calls below). The Fourier directions B
 * are fixed features and get no gradient. */
typedef struct {
  double *dW[5];
  double *db[5];
} rt_mlp_grads;

/*
 * rt_mlp_backward -- reverse mode of rt_mlp_eval: given inputs xy [n][2] and dL/d(outputs)
 * dout [n][4] (both DEVICE float32), writes dL/dW and dL/db summed over the n inputs.
 * Runs on the tensor cores: per tile of 128 inputs the forward pass is recomputed, then
 * weight gradients delta^T a (accumulated in tensor memory across all tiles of a CTA), bias
 * gradients and the delta of the layer below, with operands in the 16-bit format of
 * mlp->precision and FP32 accumulation; each CTA adds its sums to the FP64 outputs. The
 * per-input gradients are scaled by a power of two (from their largest magnitude) before
 * they are rounded to 16 bits, and the results unscaled. Scratch (pre-activations of the
 * tile in flight, 128 KiB per SM) is allocated and freed on `stream`. Returns RT_OK,
 * RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_mlp_backward(const rt_mlp *mlp, const float *xy, const float *dout, long long n,
                    const rt_mlp_grads *grads, void *stream);

/*
 * rt_render_mlp_adjoint -- rt_render_adjoint for the neural-field render of rt_render_mlp
 * (the paper trains the network by differentiating through the renderer): seeds, cube_out and
 * the grid gradients are as in rt_render_adjoint, the grid gradients being taken with respect
 * to the grid fields before the network's modulation. In addition mlp_grads receives dL/dW
 * and dL/db of the network. Steps: the network forward at every sample (as rt_render_mlp),
 * the fused march adjoint with the modulation, which also writes dL/d(outputs) per sample,
 * then rt_mlp_backward over those samples. Device buffers of 40 n_pix n_samples bytes plus
 * the scratch of both steps are allocated and freed on `stream`. Returns RT_OK, RT_EINVAL,
 * RT_ENOMEM or RT_ECUDA.
 */
int rt_render_mlp_adjoint(const rt_grid *grid, const rt_fields *fields, const rt_geom *geom,
                          const rt_view *view, const rt_line *line, const rt_mlp *mlp,
                          const float *dL_dcube, const float *target, float *cube_out,
                          const rt_grads *grads, const rt_mlp_grads *mlp_grads, void *stream);

/* rt_mlp_status -- synchronous: 1 in *timed_out if a tensor-core MMA wait ever expired in this
   process (the kernel then stops early and its outputs are incomplete), else 0. */
int rt_mlp_status(int *timed_out);

/* ------------------------------------------------------------------------------------- */
/* Serving: a continuous-batching request loop                                            */
/* ------------------------------------------------------------------------------------- */
/*
 * The paper evaluates the renderer many times over independent parameter sets (MCMC over
 * disk parameters, Methods, "MCMC Inference of HD 163296"; neural-field training steps);
 * the server below runs such independent renders and gradients as they arrive. A request is
 * admitted when the number of requests on the device is below max_inflight and its device
 * footprint fits in the memory budget (first come, first served; a request never jumps the
 * queue). Admitted requests are launched at once, each on its own stream of a pool, so that
 * the work of requests that arrive while others run overlaps on the device. Completion is
 * signalled by a host callback enqueued after the request's work; nothing waits on the
 * device. All functions are thread-safe.
 */
typedef struct rt_server rt_server;

#define RT_REQ_RENDER 0   /* rt_render */
#define RT_REQ_ADJOINT 1  /* rt_render_adjoint */

#define RT_STATE_QUEUED 0
#define RT_STATE_RUNNING 1
#define RT_STATE_DONE 2
#define RT_STATE_FAILED 3
#define RT_STATE_CANCELLED 4

#define RT_SERVER_FAKE_DEVICE 1  /* flag: run no GPU work; requests finish after fake_us */

typedef struct {
  int kind;                 /* RT_REQ_RENDER or RT_REQ_ADJOINT */
  rt_grid grid;
  rt_fields fields;         /* DEVICE fields; must stay valid until the request finishes */
  rt_geom geom;
  rt_view view;             /* v_kms (HOST) is copied at submit */
  rt_line line;
  float *cube;              /* DEVICE output [nch][ny][nx]; required for renders, may be NULL
                               for gradients */
  const float *dL_dcube;    /* gradients: exactly one of dL_dcube / target (DEVICE) */
  const float *target;
  rt_grads grads;           /* gradients: DEVICE outputs as for rt_render_adjoint */
  int fake_us;              /* RT_SERVER_FAKE_DEVICE only: simulated run time */
} rt_request;

/*
 * rt_server_create -- a server on the current device. mem_budget_bytes bounds the summed
 * footprint of the requests on the device (cube, seed and gradient buffers they touch plus
 * the scratch the adjoint allocates for gradients); max_inflight (>= 1) bounds how
 * many run at once (one stream each); max_queue (>= 1) bounds the requests waiting for
 * admission. flags: 0 or RT_SERVER_FAKE_DEVICE. Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
int rt_server_create(size_t mem_budget_bytes, int max_inflight, int max_queue, int flags,
                     rt_server **out);

/*
 * rt_submit -- validate and enqueue a request; *ticket identifies it. Returns RT_OK,
 * RT_EINVAL (malformed request, nothing enqueued), RT_ENOMEM (footprint above the whole
 * budget: it could never be admitted) or RT_EBUSY (max_queue requests already waiting).
 */
int rt_submit(rt_server *s, const rt_request *req, uint64_t *ticket);

/* rt_poll -- state of a request (RT_STATE_*) and its latency in ms: submit to completion if
   finished, submit to now otherwise. Never blocks. RT_ENOTFOUND for an unknown ticket. */
int rt_poll(rt_server *s, uint64_t ticket, int *state, double *latency_ms);

/* rt_wait -- block until the request finishes (DONE, FAILED or CANCELLED) or timeout_ms
   passes (RT_ETIMEDOUT; the request keeps running). */
int rt_wait(rt_server *s, uint64_t ticket, double timeout_ms, int *state, double *latency_ms);

/* rt_cancel -- cancel a request that is still queued (RT_OK). A running request cannot be
   cancelled (RT_EBUSY); a finished one is left as is (RT_OK). */
int rt_cancel(rt_server *s, uint64_t ticket);

/* Error message of a FAILED request ("" otherwise), copied into buf (size n). */
int rt_request_error(rt_server *s, uint64_t ticket, char *buf, size_t n);

/* Counters: requests queued and running, bytes of budget in use, requests completed. */
int rt_server_stats(rt_server *s, int *queued, int *running, size_t *bytes_in_use,
                    uint64_t *completed);

/*
 * rt_request_device_times -- when a finished request's work ran on the device (measurement
 * support; no counterpart in the paper): the times [ms] at which its stream reached the
 * points just before and just after its kernels, relative to an event the server recorded at
 * creation (CUDA events on the request's stream). Intervals of different requests that
 * intersect mean their work was in flight on the device at the same time.
 * Returns RT_OK, RT_EINVAL (null argument, fake device), RT_ENOTFOUND, RT_EBUSY (not finished)
 * or RT_ECUDA.
 */
int rt_request_device_times(rt_server *srv, uint64_t ticket, double *start_ms, double *end_ms);

/* rt_server_destroy -- cancel queued requests, wait for running ones (their device work is
   finite), release streams and the scheduler thread. */
int rt_server_destroy(rt_server *s);

/*
 * rt_pipe_peak -- measured issue rate of one arithmetic operation the march is built from,
 * for the roofline denominators of the march kernels (measurement support; the paper has no
 * counterpart). One wave of blocks (the occupancy limit x the device's SMs) runs 8
 * independent chains per thread of `op` for `iters` steps.
 *   op           RT_PEAK_* below
 *   iters        16 .. 2^24 steps per chain (2^13 takes 1-10 ms)
 *   per_s_sm     (host) results per second per SM: lanes of results completed by one SM's
 *                blocks / the CUDA-event time of the launch (packed two-lane forms count two
 *                results per lane). Divide by the SM clock sampled meanwhile for a rate per
 *                clock.
 *   ms           (host) CUDA-event time of the measured launch
 *   counter_mhz  (host) ticks of the per-SM cycle counter (clock64) per microsecond of that
 *                launch; on B300 it is not the SM clock
 * Allocates two small buffers (one entry per block) on `stream` and synchronises it.
 * Returns RT_OK, RT_EINVAL, RT_ENOMEM or RT_ECUDA.
 */
#define RT_PEAK_FFMA 0   /* fma.rn.f32 */
#define RT_PEAK_FFMA2 1  /* packed two-lane fma.rn.f32x2 (2 results per lane) */
#define RT_PEAK_EX2 2    /* ex2.approx.ftz.f32 */
#define RT_PEAK_RSQ 3    /* rsqrt.approx.ftz.f32 */
#define RT_PEAK_LG2 4    /* lg2.approx.ftz.f32 */
#define RT_PEAK_RCP 5    /* rcp.approx.ftz.f32 */
#define RT_PEAK_SQRT 6   /* sqrt.approx.ftz.f32 */
#define RT_PEAK_TANH 7   /* tanh.approx.f32 */
#define RT_PEAK_TANH2 8  /* tanh.approx.f16x2 (2 results per lane) */
int rt_pipe_peak(int op, int iters, double *per_s_sm, double *ms, double *counter_mhz,
                 void *stream);

/*
 * rt_kernel_timing / rt_kernel_time -- device time of the forward march kernel alone
 * (measurement support; no counterpart in the paper). With rt_kernel_timing(1), every forward
 * render (rt_render and the neural-field and served forwards) records a pair of CUDA events
 * on its stream around the launch of the march kernel; the march then starts after its prep
 * kernel (ray setups, corner quads) instead of overlapping its launch with it, so timed calls
 * can be a few microseconds slower. rt_kernel_time synchronises on the recorded events and
 * returns the summed milliseconds and the number of timed launches since the last read (or
 * since timing was switched on), then forgets them. rt_kernel_timing(0) stops recording and
 * drops unread pairs. Process-wide; at most 4096 pairs are kept (later launches are not
 * timed). Returns RT_OK, RT_EINVAL (null argument) or RT_ECUDA.
 */
int rt_kernel_timing(int on);
int rt_kernel_time(double *total_ms, int *launches);

/* Message for the last error on this thread ("" if none). */
const char *rt_last_error(void);

/* Library version string. */
const char *rt_version(void);

#ifdef __cplusplus
}
#endif
#endif
