/*
 * ms_oracle.h -- plain FP64 CPU oracle of the particle-continuum sea-ice model
 * (msDEM) of Deng, Stechmann & Chen, "Particle-Continuum Multiscale Modeling
 * of Sea Ice Floes" (arXiv 2303.07819).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of bench.py may load or call this library.  It shares no code, header,
 * table or helper with the CUDA library under paper_2303_07819_gb300/csrc.
 *
 * Everything is FP64, single-threaded per cell, in a fixed order:
 * pairs (l, j) with l < j in the order the floes were given (stable per cell).
 *
 * Units are SI (m, s, kg) unless a scenario chooses non-dimensional values.
 */
#ifndef MS_ORACLE_H
#define MS_ORACLE_H
#include <stdint.h>

#define ORC_NMOM 12   /* moment columns, see orc_model_moments() */
#define ORC_NWIN 5    /* window-sum columns: sum_t ubar, vbar, Fdx, Fdy, Td */
#define ORC_NCI 10    /* coarse-step inputs per cell: moment columns 1-5, window sums */

typedef struct orc_params {
    /* domain and coarse grid (one periodic DEM per coarse cell) */
    int32_t nx, ny;
    double Lx, Ly;
    /* ocean: uniform part plus stream-function Fourier modes,
     * psi = sum_m A_m sin(2 pi (kx_m X/Lx + ky_m Y/Ly) + phi_m) */
    double uo_x, uo_y;
    int32_t n_modes;
    const double *modes;           /* [n_modes][4] = A (m^2/s), kx, ky, phi (rad) */
    double rho_o, Cd;              /* ocean density, ocean drag coefficient d_o */
    double rho_a, Ca;              /* air density, wind drag coefficient */
    double wind_x, wind_y;         /* wind at t = 0 (m/s) */
    double wind_period;            /* > 0: wind vector rotates with this period (s) */
    /* ice and contact law */
    double rho_ice, E, G, eta, mu, h_ref;
    int32_t inertia_half;          /* 0: I = m r^2 (paper), 1: I = m r^2 / 2 */
    /* coupling (Algorithm 1) */
    int32_t couple, N0, n_t;
    /* ocean, second part: velocity Fourier modes (compressible currents such
     * as those of Secs. 4.2-4.3), u_o += sum_m (Au_m, Av_m) cos(kx_m X +
     * ky_m Y + phi_m) with real wave numbers (rad per unit length) */
    int32_t n_vmodes;
    const double *vmodes;          /* [n_vmodes][5] = Au, Av, kx, ky, phi */
    /* boundary in x (Sec. 4.4): 0 periodic; 1 or 2 rigid walls at X = 0 and
     * X = Lx.  The truth DEM is then not periodic in x, a floe touching a wall
     * gets the contact law of Eq. (2.2) against it (orc_wall), and a centre
     * that would pass a wall stays on it; the coarse solve has ghost cells
     * beyond the walls, zero (1) or mirrored (2) (orc_lf_bc); the per-cell
     * DEMs of the multiscale model stay doubly periodic (Sec. 3.1). */
    int32_t walls;
} orc_params;

/* ---- unit-level functions (used by the pins) ---- */
/* Ocean current, its curl and the wind at global position (X, Y), time t.
 * out = {u_o, v_o, zeta_o, u_a, v_a}. */
void orc_forcing(const orc_params *p, double X, double Y, double t, double *out);

/* Contact of floe l with floe j under periodic minimum image with periods
 * (Px, Py); a period <= 0 means no periodic image along that axis.  Returns
 * 1 if in contact.  out (16 doubles):
 * {Fx_l, Fy_l, T_l, T_j, F_normal, f_t, delta, chord, nx, ny, d, v_t, 0,0,0,0}
 * The force on j is -(Fx_l, Fy_l). */
int orc_pair(const orc_params *p, double Px, double Py,
             double xl, double yl, double ul, double vl, double wl, double rl, double hl,
             double xj, double yj, double uj, double vj, double wj, double rj, double hj,
             double *out);

/* Contact of floe l with the rigid walls X = 0 and X = Lx (Sec. 4.4).
 * reading: a wall acts as a floe at rest, without spin, of unbounded radius
 * and of at least floe l's thickness, whose edge is the wall line: the overlap
 * is delta = d - r_l with d the distance from the centre to the wall, the
 * chord of Eq. (2.2) is the chord the wall line cuts from the disk, the
 * normal points from the floe into the wall.  Returns the number of walls
 * touched (0, 1, or 2 for a floe wider than the domain).  out (16 doubles):
 * {Fx_l, Fy_l, T_l, 0, F_normal, f_t, delta, chord, nx, ny, d, v_t, 0,0,0,0},
 * forces summed over the walls, the other entries those of the last wall. */
int orc_wall(const orc_params *p, double Lx, double xl, double ul, double vl, double wl,
             double rl, double hl, double *out);

/* All contacting pairs (l < j) among n floes with periods (Px, Py).
 * Writes up to max_pairs pairs into pairs[2k], pairs[2k+1]; returns count. */
int64_t orc_contacts(const orc_params *p, double Px, double Py, int64_t n,
                     const double *x, const double *y, const double *r,
                     int64_t *pairs, int64_t max_pairs);

/* N1 Lax-Friedrichs substeps of length dtau of the moment equations on the
 * periodic coarse grid.  q = [4][ncell] (rho, rho u, rho v, P_omega), updated
 * in place; V = [2][ncell]; S = [4][ncell]. */
void orc_lf(int32_t nx, int32_t ny, double dx, double dy, double *q,
            const double *V, const double *S, double dtau, int32_t nsub);
/* The same with walls (Sec. 4.4): periodic in y only; the neighbours beyond
 * x = 0 and x = Lx are ghost cells, holding zero with walls = 1 (zero
 * Dirichlet on every field) or mirroring the boundary cell with walls = 2
 * (rho, rho v_y, P_omega equal, rho v_x and <v_x> reversed: an impermeable
 * wall).  walls = 0 is orc_lf. */
void orc_lf_bc(int32_t nx, int32_t ny, double dx, double dy, double *q,
               const double *V, const double *S, double dtau, int32_t nsub, int32_t walls);

/* ---- multiscale model (msDEM) ---- */
typedef struct orc_model orc_model;

/* Floes in global coordinates; each is assigned to the coarse cell holding its
 * centre (half-open cells) and keeps that cell for the whole run. */
orc_model *orc_model_create(const orc_params *p, int64_t n,
                            const double *x, const double *y, const double *theta,
                            const double *u, const double *v, const double *omega,
                            const double *r, const double *h);
void orc_model_free(orc_model *m);
int  orc_model_step(orc_model *m, double dt, int64_t nsteps);
/* sharded runs: hold = 1 makes orc_model_step stop right after the last fine
 * step of a coarse interval (the coarse step pending, further steps refused
 * until orc_model_coarse); the coarse inputs of every cell, [ncell][ORC_NCI]
 * = (sum m, sum m u, sum m v, sum I, sum I omega, the 5 window sums), can
 * be read and those of listed cells replaced before it runs */
void orc_model_set_hold(orc_model *m, int32_t hold);
int32_t orc_model_pending(const orc_model *m);
void orc_model_coarse_inputs(const orc_model *m, double *out);
void orc_model_set_coarse_inputs(orc_model *m, int32_t ncells, const int32_t *cells, const double *vals);
int  orc_model_coarse(orc_model *m);
/* moments of the current state: [ncell][ORC_NMOM] */
void orc_model_moments(const orc_model *m, double *out);
/* floe state in the caller's original order, global coordinates, 8 x n:
 * x, y, theta, u, v, omega, r, h */
void orc_model_floes(const orc_model *m, double *out);
/* coupling state: q [4][ncell], targets [4][ncell] (s, dvx, dvy, dw),
 * window [ORC_NWIN][ncell], flags {have_q, have_targets, steps_done} */
void orc_model_coupling(const orc_model *m, double *q, double *targets,
                        double *window, int64_t *flags);
/* per-cell floe offsets (ncell+1) and original index of each stored floe */
void orc_model_layout(const orc_model *m, int64_t *off, int64_t *orig);

/* ---- truth model: one DEM over the whole periodic domain ---- */
typedef struct orc_truth orc_truth;
orc_truth *orc_truth_create(const orc_params *p, int64_t n,
                            const double *x, const double *y, const double *theta,
                            const double *u, const double *v, const double *omega,
                            const double *r, const double *h);
void orc_truth_free(orc_truth *t);
int  orc_truth_step(orc_truth *t, double dt, int64_t nsteps);
/* brute = 1: contact forces by the plain loop over all pairs (l < j); 0 (the
 * default): the same pairs found through bins of side >= 2 r_max, summed in
 * the same order, so the result is identical bit for bit. */
void orc_truth_set_brute(orc_truth *t, int32_t brute);
void orc_truth_moments(const orc_truth *t, double *out);
void orc_truth_floes(const orc_truth *t, double *out);

/* L2 norm of the difference of two cell fields (Sec. 4.1). */
double orc_l2_diff(int32_t nx, int32_t ny, double dx, double dy,
                   const double *a, const double *b);

void orc_set_threads(int32_t nthreads);
int32_t orc_get_threads(void);

#endif
