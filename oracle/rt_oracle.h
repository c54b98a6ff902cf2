/*
 * FP64 CPU oracle for the line radiative-transfer march (TEST INFRASTRUCTURE ONLY).
 *
 * This library is the slow, plain, double-precision statement of what the GPU path
 * computes. Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
 * load it; the product path never links, loads or calls it, and it shares no code, header,
 * table or constant with the CUDA library.
 *
 * Physics followed (arXiv 2509.03623, Methods):
 *   - integral form of the transfer equation, Eq. rt-int, with the optical depth of
 *     Eq. optical_depth, traced backward from each image pixel;
 *   - emissivity j_nu and extinction beta_nu from the level populations and Einstein
 *     coefficients (the two equations following Eq. optical_depth);
 *   - LTE (Boltzmann) level populations;
 *   - the Doppler-shifted Gaussian line profile phi(nu) with delta_nu = omega.v / c;
 *   - the line width alpha(x) (thermal + turbulent) and sound speed c_s;
 *   - the Keplerian term of Eq. gas_velocity_pressure.
 * Readings where the paper is silent are listed in the design notes and repeated at the
 * point of use below.
 */
#ifndef RT_ORACLE_H
#define RT_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

/* General 3-D Cartesian node grid in the disk frame (the RadJAX setting beyond the
   axisymmetric disk): nodes uniformly spaced over [x0, x1] x [y0, y1] x [z0, z1] au, fields
   [nz][ny][nx] (x fastest): T [K], n_H2 [cm^-3], v_turb [km/s or Mach], X_CO (abundance),
   gas velocity (vx, vy, vz) [km/s]; trilinear interpolation, nothing outside the box. */
typedef struct {
  int nx, ny, nz;
  double x0, x1, y0, y1, z0, z1;
  const double *T, *n_h2, *vturb, *x_co, *vx, *vy, *vz;
} orc_grid3;

/* 3-D spherical node grid centred on the star (the grid of the paper's runtime benchmark):
   r log-spaced (r_log=1) or linear (r_log=0) in [r_in, r_out] au; colatitude theta (angle
   from +z) linear in [th0, th1] rad; azimuth phi = atan2(y, x) in [0, 2 pi) with nph nodes at
   2 pi k / nph, periodic. Fields [nph][nth][nr] (r fastest): T [K], n_H2 [cm^-3], v_turb,
   X_CO, and the gas velocity in spherical components (v_r, v_theta, v_phi) [km/s]; trilinear
   interpolation in (radial index, theta, phi); no gas outside r_in <= r <= r_out,
   th0 <= theta <= th1. Rays are sampled over their chord through the sphere r <= r_out. */
typedef struct {
  int nr, nth, nph, r_log;
  double r_in, r_out, th0, th1;
  const double *T, *n_h2, *vturb, *x_co, *vr, *vth, *vph;
} orc_grid_sph;

typedef struct {
  /* (r, z/r) node grid: r log-spaced (r_log=1) or linear (r_log=0) in [r_in, r_out] au,
     z/r linear in [0, zr_max]. */
  int nr, nz, r_log;
  double r_in_au, r_out_au, zr_max;
  /* node fields, [nz][nr] row-major: T [K], n_H2 [cm^-3], v_turb [km/s, or Mach number
     when vturb_mach=1]; surfaces h_lo, h_hi [nr] in z/r units. */
  const double *T, *n_h2, *vturb, *h_lo, *h_hi;
  double x_co, edge_w;
  int vturb_mach;
  /* geometry */
  double incl_deg, pa_deg, dist_pc, mstar_msun, vsys_kms;
  /* image and spectral sampling */
  int nx, ny;
  double half_fov_au;
  int nch;
  const double *v_kms;
  int n_samples;
  double I0;
  int units; /* 0: erg s^-1 cm^-2 Hz^-1 sr^-1, 1: Jy per pixel */
  /* line (rigid rotor, J_u -> J_u-1) */
  double nu0_hz, A_ul, B_rot_hz, m_co_amu, m_mol_amu;
  int J_u;
  /* optional rotation field [nz][nr] in km/s (Eq. gas_velocity_pressure with the pressure
     term, e.g. from orc_pressure_vphi), interpolated like the other node fields; NULL: the
     Keplerian term alone, evaluated exactly at each point */
  const double *vphi;
  /* optional 3-D grid: when set, the node grid, fields, surfaces, rotation and stellar mass
     above are not used; rays are clipped to the box (rt_render3d's sampling rule) */
  const orc_grid3 *g3;
  /* optional spherical grid (used like g3 when set; g3 must then be NULL) */
  const orc_grid_sph *gs;
} orc_problem;

/* Full cube [nch][ny][nx]. Returns 0, or -1 on invalid arguments. */
int orc_render(const orc_problem *p, double *cube, int nthreads);

/* Spectra of selected pixels: pix[i] = iy*nx + ix; out [npix][nch]. */
int orc_render_pixels(const orc_problem *p, const long long *pix, int npix, double *out,
                      int nthreads);

/* Ray chord through the bounding cylinder: returns 1 and fills s_in, s_out (au along the
   ray, origin on the sky plane through the star) and the ray origin/direction, or 0 on a
   miss. */
int orc_ray(const orc_problem *p, int ix, int iy, double *s_in, double *s_out, double *P0,
            double *omega);

/* Local quantities at a disk-frame point (au) for channel velocity v_kms:
   out[0]=j_nu, out[1]=beta_nu (cgs), out[2]=T, out[3]=n_H2, out[4]=X_CO, out[5]=v_los [km/s],
   out[6]=alpha [km/s], out[7]=n_u, out[8]=n_l, out[9]=phi [Hz^-1], out[10]=S=j/beta,
   out[11]=v_turb (input units). Returns 1 if gas is present, 0 otherwise. */
int orc_point(const orc_problem *p, double x, double y, double z, double v_kms, double *out);

/* Rigid-rotor partition function Z(T) = sum_J (2J+1) exp(-h B J(J+1) / kT). */
double orc_partition(double T, double B_rot_hz);

/* Reverse-mode gradient of a scalar loss L given dL/dcube [nch][ny][nx] (cube units).
   Writes the cube and dL/d(node fields) [nz][nr] and dL/d(surfaces) [nr]; every gradient
   array is overwritten. */
int orc_render_adjoint(const orc_problem *p, const double *dL_dcube, double *cube,
                       double *dT, double *dn, double *dvt, double *dh_lo, double *dh_hi,
                       int nthreads);

/* orc_render_adjoint for a problem with a rotation field (p->vphi): also writes
   dL/d(rotation field) [nz][nr] (per km/s, overwritten) through
   v_los = v_phi (omega . phi^) + v_sys with the field interpolated bilinearly. */
int orc_render_adjoint_vphi(const orc_problem *p, const double *dL_dcube, double *cube,
                            double *dT, double *dn, double *dvt, double *dh_lo, double *dh_hi,
                            double *dvphi, int nthreads);

/* Reverse mode of the 3-D grid marches (exactly one of p->g3, p->gs set): given dL/dcube
   [nch][ny][nx], writes the cube and dL/d(node fields) in the grid's node order ([nz][ny][nx]
   Cartesian, [nph][nth][nr] spherical) for T, n_H2, v_turb, the CO abundance and the three
   velocity fields (dvx, dvy, dvz receive v_x, v_y, v_z or v_r, v_theta, v_phi; per km/s); every
   gradient array is overwritten. The hand-derived reverse of the same per-sample loop as
   orc_render_adjoint, with the trilinear weights in place of the bilinear ones. */
int orc_render_adjoint3(const orc_problem *p, const double *dL_dcube, double *cube, double *dT,
                        double *dn, double *dvt, double *dxco, double *dvx, double *dvy,
                        double *dvz, int nthreads);

/* Neural field (fully connected, SiLU hidden activations, Fourier-feature input). */
typedef struct {
  int n_freq;              /* number of Fourier directions; features = 2*n_freq */
  const double *B;         /* [n_freq][2] frequencies applied to (rhat, zhat) */
  int n_layers;            /* number of Linear layers (hidden layers + output layer) */
  const int *dims;         /* [n_layers+1]: dims[0] = 2*n_freq, ..., dims[n_layers] = outputs */
  const double *const *W;  /* W[l]: [dims[l+1]][dims[l]] row-major */
  const double *const *b;  /* b[l]: [dims[l+1]] */
  double h_scale;          /* surface offset scale applied to outputs 2 and 3 */
} orc_mlp;

/* Network outputs for npts inputs x[i] = (rhat, zhat): out [npts][dims[n_layers]]. */
int orc_mlp_eval(const orc_mlp *m, const double *x, int npts, double *out);

/* Reverse mode of orc_mlp_eval: dL/dW and dL/db (flat, layer after layer as in
   orc_render_mlp_adjoint; overwritten) summed over npts inputs x with output gradients
   gout [npts][dims[n_layers]]. */
int orc_mlp_grad(const orc_mlp *m, const double *x, const double *gout, int npts, double *dW,
                 double *db);

/* Cube rendered with the neural field: at every sample the grid values are modulated by the
   network outputs o: T <- T exp(o0), n <- n exp(o1), h_lo <- h_lo + h_scale o2,
   h_hi <- h_hi + h_scale o3. pix/npix select pixels as in orc_render_pixels (pix=NULL: all,
   out is then the full cube [nch][ny][nx]). */
int orc_render_mlp(const orc_problem *p, const orc_mlp *m, const long long *pix, int npix,
                   double *out, int nthreads);

/* Reverse mode of orc_render_mlp for the full cube: as orc_render_adjoint (node gradients are
   with respect to the grid fields before the network modulation), plus dL/dW and dL/db of the
   network, flat in layer order (layer l: [dims[l+1]][dims[l]] and [dims[l+1]]). Every
   gradient array is overwritten. The Fourier directions B are not differentiated. */
int orc_render_mlp_adjoint(const orc_problem *p, const orc_mlp *m, const double *dL_dcube,
                           double *cube, double *dT, double *dn, double *dvt, double *dh_lo,
                           double *dh_hi, double *dW, double *db, int nthreads);

/* Physics-constrained field chain (Methods, "Parametric Disk Modeling": Eq. gas_density_temp,
   the surface-density profile Sigma(r), Eq. column_density and Eq. co_layer; applied to a
   temperature grid as in "Neural Temperature Recovery", physics-informed constraints).
   Per radius node r_i, on the nodes z_j = w_j r_i (w_j = j zr_max / (nz - 1)):
     d ln rho / dz = -G M z m_mol / ((r^2 + z^2)^{3/2} k T) - d ln T / dz, integrated upward
       from the midplane with the trapezoid rule on the nodes (the ln T term exactly);
     rho normalised so that 2 int_0^{z_max} rho dz (trapezoid, mirror symmetry) = Sigma(r),
       Sigma(r) = Sigma0 (r/r_c)^-gamma exp(-(r/r_c)^{2 - gamma});
     n_H2 = rho / m_mol;  N_H2(z_j) = int_{z_j}^{z_max} n_H2 dz (trapezoid);
     CO where T > T_freeze and 0.706 N_H2 > N_dissoc, returned as the two surfaces of the
     layer in z/r: h_lo = lowest w with T > T_freeze (T linear between nodes; 0 if the
     midplane node is warmer, zr_max if no node is), h_hi = highest w with
     0.706 N_H2 > N_dissoc (N_H2 linear between nodes; 0 if no node qualifies).
   Uses p->nr, nz, r_log, r_in_au, r_out_au, zr_max, mstar_msun, m_mol_amu. Outputs
   n_h2, N_h2 [nz][nr] (cm^-3, cm^-2; N_h2 may be NULL), h_lo, h_hi [nr]. */
typedef struct {
  double sigma0_gcm2, r_c_au, gamma;
  double T_freeze, N_dissoc_cm2;
} orc_chain;

int orc_field_chain(const orc_problem *p, const orc_chain *c, const double *T, double *n_h2,
                    double *N_h2, double *h_lo, double *h_hi);

/* Reverse mode of orc_field_chain for a scalar loss L: from dL/dn_h2 [nz][nr] and dL/dh_lo,
   dL/dh_hi [nr] (any of them NULL: zero) writes dL/dT [nz][nr] (overwritten), through the
   hydrostatic integration and its normalisation (n_H2), the column N_H2 (h_hi) and the
   freeze-out crossing (h_lo). A surface depends on the two nodes of the cell where its
   threshold is crossed, through the linear interpolation inside that cell (the choice of the
   cell is piecewise constant in T); a surface pinned at 0 or zr_max has zero derivative. */
int orc_field_chain_adjoint(const orc_problem *p, const orc_chain *c, const double *T,
                            const double *g_n, const double *g_lo, const double *g_hi,
                            double *g_T);

/* Pressure-corrected rotation on the nodes (Eq. gas_velocity_pressure):
     v_phi^2 = G M r^2 / (r^2 + z^2)^{3/2} + (r / rho) dP/dr |_z,  P = n_H2 k T,  rho = m_mol n_H2,
   with dP/dr at constant z from the grid coordinates (u = ln r or r, w = z/r):
     dP/dr |_z = (du/dr) dP/du |_w - (w / r) dP/dw |_u,
   each derivative a second-order central difference (second-order one-sided at the first and
   last node; first-order when the axis has two nodes). v_phi^2 < 0 (pressure support beyond
   gravity) gives v_phi = 0; a node without gas (n_H2 = 0) keeps the Keplerian term. Uses
   p->nr, nz, r_log, r_in_au, r_out_au, zr_max, mstar_msun, m_mol_amu. vphi [nz][nr] km/s. */
int orc_pressure_vphi(const orc_problem *p, const double *n_h2, const double *T, double *vphi);

/* Reverse mode of orc_pressure_vphi for a scalar loss L: from dL/dvphi [nz][nr] (per km/s)
   writes dL/dn_h2 and dL/dT [nz][nr] (overwritten) through the pressure term (the difference
   stencils transposed and the 1/rho factor); nodes clamped to v_phi = 0 and nodes without gas
   (Keplerian term only) contribute nothing. */
int orc_pressure_vphi_adjoint(const orc_problem *p, const double *n_h2, const double *T,
                              const double *g_v, double *g_n, double *g_T);

#ifdef __cplusplus
}
#endif
#endif
