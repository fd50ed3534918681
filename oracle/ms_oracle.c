/*
 * ms_oracle.c -- plain FP64 CPU oracle of the msDEM particle-continuum model
 * (Deng, Stechmann & Chen, arXiv 2303.07819).
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, the smoke check and the CPU
 * baseline of bench.py; never by the product path.  Shares no code with the
 * CUDA library.
 *
 * Written for a reader to check against the paper by eye:
 *   - DEM of disk floes: Sec. 2.1, Eq. (2.1a-d) and the contact law Eq. (2.2);
 *   - forward Euler in time: Sec. 3.1;
 *   - one doubly periodic DEM per coarse cell: Sec. 3.1 (superparameterization);
 *   - moments rho, rho v, P_omega: Sec. 2.3, Eq. (2.26a-c), with the Oseen
 *     linearisation of Eq. (3.3), solved by Lax-Friedrichs (Sec. 3.2);
 *   - coupling schedule: Algorithm 1; gradual updates: Sec. 3.3, Eqs. (3.4-3.7).
 * Readings of the places where the paper is silent or garbled are noted inline
 * ("reading:").
 */
#include "ms_oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const double PI = 3.14159265358979323846;
static int32_t g_threads = 1;

void orc_set_threads(int32_t nthreads) { g_threads = nthreads > 0 ? nthreads : 1; }
int32_t orc_get_threads(void) { return g_threads; }

/* ------------------------------------------------------------------ forcing */

/* Wind: the paper adds wind "by similar terms to the ocean drag" (Sec. 2.1).
 * reading: a time-varying wind rotates the t = 0 vector at a constant rate. */
static void wind_at(const orc_params *p, double t, double *ua, double *va)
{
    if (p->wind_period > 0.0) {
        double ang = 2.0 * PI * t / p->wind_period;
        double c = cos(ang), s = sin(ang);
        *ua = p->wind_x * c - p->wind_y * s;
        *va = p->wind_x * s + p->wind_y * c;
    } else {
        *ua = p->wind_x;
        *va = p->wind_y;
    }
}

/* Ocean velocity u_o = (-dpsi/dy, dpsi/dx) + uniform part, and its curl
 * (curl u_o = laplacian psi), which enters the rotational drag of Eq. (2.1d). */
void orc_forcing(const orc_params *p, double X, double Y, double t, double *out)
{
    double uo = p->uo_x, vo = p->uo_y, zeta = 0.0;
    for (int32_t m = 0; m < p->n_modes; m++) {
        const double *md = p->modes + 4 * m;
        double A = md[0];
        double kx = 2.0 * PI * md[1] / p->Lx;
        double ky = 2.0 * PI * md[2] / p->Ly;
        double th = kx * X + ky * Y + md[3];
        double c = cos(th), s = sin(th);
        uo -= A * ky * c;
        vo += A * kx * c;
        zeta -= A * (kx * kx + ky * ky) * s;
    }
    /* velocity modes: u += Au cos(th), v += Av cos(th), so the curl
     * dv/dx - du/dy adds -(Av kx - Au ky) sin(th) */
    for (int32_t m = 0; m < p->n_vmodes; m++) {
        const double *md = p->vmodes + 5 * m;
        double th = md[2] * X + md[3] * Y + md[4];
        double c = cos(th), s = sin(th);
        uo += md[0] * c;
        vo += md[1] * c;
        zeta -= (md[1] * md[2] - md[0] * md[3]) * s;
    }
    double ua, va;
    wind_at(p, t, &ua, &va);
    out[0] = uo; out[1] = vo; out[2] = zeta; out[3] = ua; out[4] = va;
}

/* ------------------------------------------------------------ contact law */

/* Contact of floe l with floe j, Eq. (2.2) with the Coulomb limit of Sec. 2.1.
 * reading: n points from l to j and delta = d - (r_l + r_j) < 0 in overlap, so
 * f_n = c E delta n pushes l away from j; the normal law carries an optional
 * dashpot eta; thickness enters as min(h_l, h_j)/h_ref (the paper's floes
 * have unit thickness); the tangential law is viscous in v_t; torques are
 * r_l f_t on l and r_j f_t on j (Eq. 2.1d, r^j points from j towards l). */
int orc_pair(const orc_params *p, double Px, double Py,
             double xl, double yl, double ul, double vl, double wl, double rl, double hl,
             double xj, double yj, double uj, double vj, double wj, double rj, double hj,
             double *out)
{
    double dx = xj - xl, dy = yj - yl;
    /* periodic minimum image (none along an axis with a wall) */
    if (Px > 0.0) dx -= Px * rint(dx / Px);
    if (Py > 0.0) dy -= Py * rint(dy / Py);
    double d = sqrt(dx * dx + dy * dy);
    double sum_r = rl + rj;
    for (int k = 0; k < 16; k++) out[k] = 0.0;
    out[10] = d;
    /* nonzero only in contact (Sec. 2.1); d = 0 has no normal direction */
    if (!(d > 0.0 && d < sum_r)) return 0;
    double nx = dx / d, ny = dy / d;
    double tx = -ny, ty = nx;                 /* t = z x n */
    double delta = d - sum_r;
    /* chord length of the overlap lens; a floe inside the other: smaller diameter */
    double chord;
    if (d <= fabs(rl - rj)) {
        chord = 2.0 * fmin(rl, rj);
    } else {
        double a = (d * d + rl * rl - rj * rj) / (2.0 * d);
        double c2 = rl * rl - a * a;
        chord = 2.0 * sqrt(c2 > 0.0 ? c2 : 0.0);
    }
    double hc = fmin(hl, hj) / p->h_ref;
    double dux = uj - ul, duy = vj - vl;
    double vn = dux * nx + duy * ny;
    double Fn = chord * hc * (p->E * delta + p->eta * vn);
    if (Fn > 0.0) Fn = 0.0;                   /* contacts never attract */
    /* relative velocity of the contact points along t */
    double vt = dux * tx + duy * ty - wj * rj - wl * rl;
    double ft = chord * hc * p->G * vt;
    double cap = p->mu * fabs(Fn);            /* |f_t| <= mu |f_n| */
    if (ft > cap) ft = cap;
    else if (ft < -cap) ft = -cap;
    out[0] = Fn * nx + ft * tx;
    out[1] = Fn * ny + ft * ty;
    out[2] = rl * ft;
    out[3] = rj * ft;
    out[4] = Fn;
    out[5] = ft;
    out[6] = delta;
    out[7] = chord;
    out[8] = nx;
    out[9] = ny;
    out[11] = vt;
    return 1;
}

/* Floe l against the walls X = 0 and X = Lx (Sec. 4.4), the law of
 * orc_pair with the wall as partner: at rest, no spin, thickness >= h_l, and
 * its boundary the straight wall line, so the overlap lens becomes the
 * circular segment the line cuts off and its chord 2 sqrt(r^2 - d^2). */
int orc_wall(const orc_params *p, double Lx, double xl, double ul, double vl, double wl,
             double rl, double hl, double *out)
{
    for (int k = 0; k < 16; k++) out[k] = 0.0;
    int touched = 0;
    for (int side = 0; side < 2; side++) {
        /* the normal n points from the floe into the wall */
        double d = side == 0 ? xl : Lx - xl;
        double nx = side == 0 ? -1.0 : 1.0, ny = 0.0;
        if (!(d < rl)) continue;
        double tx = -ny, ty = nx;
        double delta = d - rl;
        double chord = d > -rl ? 2.0 * sqrt(rl * rl - d * d) : 2.0 * rl;
        double hc = hl / p->h_ref;
        double dux = -ul, duy = -vl;              /* wall velocity minus floe velocity */
        double vn = dux * nx + duy * ny;
        double Fn = chord * hc * (p->E * delta + p->eta * vn);
        if (Fn > 0.0) Fn = 0.0;
        double vt = dux * tx + duy * ty - wl * rl;
        double ft = chord * hc * p->G * vt;
        double cap = p->mu * fabs(Fn);
        if (ft > cap) ft = cap;
        else if (ft < -cap) ft = -cap;
        out[0] += Fn * nx + ft * tx;
        out[1] += Fn * ny + ft * ty;
        out[2] += rl * ft;
        out[4] = Fn; out[5] = ft; out[6] = delta; out[7] = chord;
        out[8] = nx; out[9] = ny; out[10] = d; out[11] = vt;
        touched++;
    }
    return touched;
}

int64_t orc_contacts(const orc_params *p, double Px, double Py, int64_t n,
                     const double *x, const double *y, const double *r,
                     int64_t *pairs, int64_t max_pairs)
{
    int64_t cnt = 0;
    double o[16];
    for (int64_t l = 0; l < n; l++)
        for (int64_t j = l + 1; j < n; j++) {
            if (orc_pair(p, Px, Py, x[l], y[l], 0, 0, 0, r[l], 1.0,
                         x[j], y[j], 0, 0, 0, r[j], 1.0, o)) {
                if (cnt < max_pairs) { pairs[2 * cnt] = l; pairs[2 * cnt + 1] = j; }
                cnt++;
            }
        }
    return cnt;
}

/* ------------------------------------------------------- per-floe physics */

static double floe_mass(const orc_params *p, double r, double h)
{
    return p->rho_ice * PI * r * r * h;      /* Sec. 2.1, thickness h */
}

static double floe_inertia(const orc_params *p, double m, double r)
{
    return (p->inertia_half ? 0.5 : 1.0) * m * r * r;   /* paper: I = m r^2 */
}

/* Ocean and wind drag, Eq. (2.1c-d): alpha = d_o rho_o pi r^2,
 * beta = d_o rho_o pi r^4; wind drag has the ocean's form (reading). */
static void drag(const orc_params *p, const double *f, double u, double v,
                 double w, double r, double *Fx, double *Fy, double *T)
{
    double alpha_o = p->Cd * p->rho_o * PI * r * r;
    double alpha_a = p->Ca * p->rho_a * PI * r * r;
    double beta_o = p->Cd * p->rho_o * PI * r * r * r * r;
    double du = f[0] - u, dv = f[1] - v;
    double s_o = sqrt(du * du + dv * dv);
    double au = f[3] - u, av = f[4] - v;
    double s_a = sqrt(au * au + av * av);
    double dw = 0.5 * f[2] - w;
    *Fx = alpha_o * du * s_o + alpha_a * au * s_a;
    *Fy = alpha_o * dv * s_o + alpha_a * av * s_a;
    *T = beta_o * dw * fabs(dw);
}

/* ------------------------------------------------------------- LF solver */

/* Lax-Friedrichs on the periodic coarse grid (Sec. 3.2).
 * reading: 2-D LF with the four-neighbour average; rho and P_omega in the
 * conservative form of Eq. (2.26a,c); rho v in the Oseen form of Eq. (3.3),
 * <v> . grad(rho v) with <v> taken at the cell itself.
 * Walls (Sec. 4.4): a neighbour beyond x = 0 or x = Lx is a ghost cell.
 * walls = 1, zero Dirichlet as the paper states it: the ghost's fields, and so
 * its fluxes, are zero.  walls = 2, impermeable wall: the ghost mirrors the
 * boundary cell (rho, rho v_y, P_omega equal, rho v_x and <v_x> of opposite
 * sign), so neither the flux nor the averaging moves mass through the wall. */
void orc_lf_bc(int32_t nx, int32_t ny, double dx, double dy, double *q,
               const double *V, const double *S, double dtau, int32_t nsub, int32_t walls)
{
    int64_t nc = (int64_t)nx * ny;
    double *qn = (double *)malloc(sizeof(double) * 4 * nc);
    const double *Vx = V, *Vy = V + nc;
    for (int32_t k = 0; k < nsub; k++) {
        for (int32_t j = 0; j < ny; j++)
            for (int32_t i = 0; i < nx; i++) {
                int64_t c = (int64_t)j * nx + i;
                int64_t cE = (int64_t)j * nx + (i + 1) % nx;
                int64_t cW = (int64_t)j * nx + (i + nx - 1) % nx;
                int64_t cN = (int64_t)((j + 1) % ny) * nx + i;
                int64_t cS = (int64_t)((j + ny - 1) % ny) * nx + i;
                int ghostE = walls && i == nx - 1, ghostW = walls && i == 0;
                for (int f = 0; f < 4; f++) {
                    const double *g = q + f * nc;
                    /* ghost value and ghost <v_x> */
                    double sg = f == 1 ? -1.0 : 1.0;
                    double gG = walls == 2 ? sg * g[c] : 0.0, VG = walls == 2 ? -Vx[c] : 0.0;
                    double gE = ghostE ? gG : g[cE], gW = ghostW ? gG : g[cW];
                    double VE = ghostE ? VG : Vx[cE], VW = ghostW ? VG : Vx[cW];
                    double avg = 0.25 * ((gE + gW) + (g[cN] + g[cS]));
                    double val;
                    if (f == 0 || f == 3) {
                        val = avg - dtau / (2.0 * dx) * (VE * gE - VW * gW)
                                  - dtau / (2.0 * dy) * (Vy[cN] * g[cN] - Vy[cS] * g[cS]);
                    } else {
                        val = avg - dtau * Vx[c] / (2.0 * dx) * (gE - gW)
                                  - dtau * Vy[c] / (2.0 * dy) * (g[cN] - g[cS]);
                    }
                    qn[f * nc + c] = val + dtau * S[f * nc + c];
                }
            }
        memcpy(q, qn, sizeof(double) * 4 * nc);
    }
    free(qn);
}

void orc_lf(int32_t nx, int32_t ny, double dx, double dy, double *q,
            const double *V, const double *S, double dtau, int32_t nsub)
{
    orc_lf_bc(nx, ny, dx, dy, q, V, S, dtau, nsub, 0);
}

/* ------------------------------------------------------------ msDEM model */

struct orc_model {
    orc_params p;
    double *modes;
    int64_t n;
    int32_t ncell;
    double dx, dy;                 /* coarse cell sides = periods of each DEM */
    int64_t *off, *orig;
    double *x, *y, *th, *u, *v, *w, *r, *h;   /* x, y local to the cell */
    double *fx, *fy, *tq;          /* force accumulators */
    double *fdx, *fdy, *tdq;       /* this step's drag, for the moments */
    double *r0;                    /* radius snapshot at the last coarse step */
    double *mom;                   /* [ncell][ORC_NMOM] */
    double *win;                   /* [ORC_NWIN][ncell] */
    double *q;                     /* [4][ncell] coarse state */
    double *tgt;                   /* [4][ncell] s, dvx, dvy, dw */
    int have_q, have_tgt;
    int64_t steps;
    double dt;
    int hold_coarse;               /* stop before each coarse step (sharded runs) */
    int coarse_pending;
};

/* copy of the parameters with both mode tables in one owned buffer */
static void copy_params(orc_params *dst, double **modes, const orc_params *src)
{
    *dst = *src;
    *modes = NULL;
    const int32_t ns = src->n_modes > 0 ? src->n_modes : 0, nv = src->n_vmodes > 0 ? src->n_vmodes : 0;
    if (ns + nv > 0) {
        *modes = (double *)malloc(sizeof(double) * (4 * ns + 5 * nv));
        if (ns) memcpy(*modes, src->modes, sizeof(double) * 4 * ns);
        if (nv) memcpy(*modes + 4 * ns, src->vmodes, sizeof(double) * 5 * nv);
    }
    dst->n_modes = ns;
    dst->n_vmodes = nv;
    dst->modes = ns ? *modes : NULL;
    dst->vmodes = nv ? *modes + 4 * ns : NULL;
}

static int32_t cell_index(double X, double L, double d, int32_t n)
{
    double Xw = X - L * floor(X / L);
    int32_t i = (int32_t)floor(Xw / d);
    if (i < 0) i = 0;
    if (i > n - 1) i = n - 1;
    return i;
}

/* moments of one cell of the msDEM model from the current state and the
 * stored drag of the last step: see orc_model_moments(). */
static void cell_moments(const orc_params *p, int64_t b, int64_t e,
                         const double *u, const double *v, const double *w,
                         const double *r, const double *h, const double *fdx,
                         const double *fdy, const double *tdq, double *mo)
{
    for (int k = 0; k < ORC_NMOM; k++) mo[k] = 0.0;
    for (int64_t l = b; l < e; l++) {
        double m = floe_mass(p, r[l], h[l]);
        double I = floe_inertia(p, m, r[l]);
        mo[0] += 1.0;
        mo[1] += m;
        mo[2] += m * u[l];
        mo[3] += m * v[l];
        mo[4] += I;
        mo[5] += I * w[l];
        mo[6] += PI * r[l] * r[l];
        mo[7] += m * u[l] * u[l];
        mo[8] += m * v[l] * v[l];
        mo[9] += fdx[l];
        mo[10] += fdy[l];
        mo[11] += tdq[l];
    }
}

orc_model *orc_model_create(const orc_params *p, int64_t n,
                            const double *x, const double *y, const double *theta,
                            const double *u, const double *v, const double *omega,
                            const double *r, const double *h)
{
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    copy_params(&m->p, &m->modes, p);
    m->n = n;
    m->ncell = p->nx * p->ny;
    m->dx = p->Lx / p->nx;
    m->dy = p->Ly / p->ny;
    int32_t nc = m->ncell;
    m->off = (int64_t *)calloc(nc + 1, sizeof(int64_t));
    m->orig = (int64_t *)malloc(sizeof(int64_t) * (n > 0 ? n : 1));
    double **arrs[] = {&m->x, &m->y, &m->th, &m->u, &m->v, &m->w, &m->r, &m->h,
                       &m->fx, &m->fy, &m->tq, &m->fdx, &m->fdy, &m->tdq, &m->r0};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); k++)
        *arrs[k] = (double *)calloc(n > 0 ? n : 1, sizeof(double));
    m->mom = (double *)calloc((size_t)nc * ORC_NMOM, sizeof(double));
    m->win = (double *)calloc((size_t)nc * ORC_NWIN, sizeof(double));
    m->q = (double *)calloc((size_t)nc * 4, sizeof(double));
    m->tgt = (double *)calloc((size_t)nc * 4, sizeof(double));

    /* stable assignment of floes to the cell holding their centre */
    int32_t *cid = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (int64_t l = 0; l < n; l++) {
        int32_t ix = cell_index(x[l], p->Lx, m->dx, p->nx);
        int32_t iy = cell_index(y[l], p->Ly, m->dy, p->ny);
        cid[l] = iy * p->nx + ix;
        m->off[cid[l] + 1]++;
    }
    for (int32_t c = 0; c < nc; c++) m->off[c + 1] += m->off[c];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * nc);
    for (int32_t c = 0; c < nc; c++) fill[c] = m->off[c];
    for (int64_t l = 0; l < n; l++) {
        int32_t c = cid[l];
        int64_t k = fill[c]++;
        int32_t ix = c % p->nx, iy = c / p->nx;
        double Xw = x[l] - p->Lx * floor(x[l] / p->Lx);
        double Yw = y[l] - p->Ly * floor(y[l] / p->Ly);
        m->orig[k] = l;
        m->x[k] = Xw - ix * m->dx;           /* position local to the cell */
        m->y[k] = Yw - iy * m->dy;
        m->th[k] = theta[l];
        m->u[k] = u[l];
        m->v[k] = v[l];
        m->w[k] = omega[l];
        m->r[k] = r[l];
        m->h[k] = h[l];
    }
    free(fill);
    free(cid);
    for (int32_t c = 0; c < nc; c++)
        cell_moments(&m->p, m->off[c], m->off[c + 1], m->u, m->v, m->w, m->r, m->h,
                     m->fdx, m->fdy, m->tdq, m->mom + (size_t)c * ORC_NMOM);
    return m;
}

void orc_model_free(orc_model *m)
{
    if (!m) return;
    double *arrs[] = {m->x, m->y, m->th, m->u, m->v, m->w, m->r, m->h, m->fx, m->fy,
                      m->tq, m->fdx, m->fdy, m->tdq, m->r0, m->mom, m->win, m->q,
                      m->tgt, m->modes};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); k++) free(arrs[k]);
    free(m->off);
    free(m->orig);
    free(m);
}

/* One fine step of the DEM of one cell (Eq. 2.1, forward Euler), then the
 * gradual update if this step is an update step, then the cell's moments. */
static void model_cell_step(orc_model *m, int32_t c, double dt, double t,
                            int ramp, double ramp_frac)
{
    const orc_params *p = &m->p;
    int64_t b = m->off[c], e = m->off[c + 1];
    int32_t ix = c % p->nx, iy = c / p->nx;
    double X0 = ix * m->dx, Y0 = iy * m->dy;
    double o[16];
    for (int64_t l = b; l < e; l++) { m->fx[l] = 0.0; m->fy[l] = 0.0; m->tq[l] = 0.0; }
    /* contacts: every pair of the cell once, periodic over the cell */
    for (int64_t l = b; l < e; l++)
        for (int64_t j = l + 1; j < e; j++) {
            if (orc_pair(p, m->dx, m->dy,
                         m->x[l], m->y[l], m->u[l], m->v[l], m->w[l], m->r[l], m->h[l],
                         m->x[j], m->y[j], m->u[j], m->v[j], m->w[j], m->r[j], m->h[j], o)) {
                m->fx[l] += o[0]; m->fy[l] += o[1]; m->tq[l] += o[2];
                m->fx[j] -= o[0]; m->fy[j] -= o[1]; m->tq[j] += o[3];
            }
        }
    /* drag at the floe's global position (reading: cell origin + local) */
    for (int64_t l = b; l < e; l++) {
        double f[5], Fx, Fy, T;
        orc_forcing(p, X0 + m->x[l], Y0 + m->y[l], t, f);
        drag(p, f, m->u[l], m->v[l], m->w[l], m->r[l], &Fx, &Fy, &T);
        m->fdx[l] = Fx; m->fdy[l] = Fy; m->tdq[l] = T;
        m->fx[l] += Fx; m->fy[l] += Fy; m->tq[l] += T;
    }
    /* forward Euler: every right-hand side at t_n */
    for (int64_t l = b; l < e; l++) {
        double ms = floe_mass(p, m->r[l], m->h[l]);
        double I = floe_inertia(p, ms, m->r[l]);
        m->x[l] += dt * m->u[l];
        m->y[l] += dt * m->v[l];
        m->th[l] += dt * m->w[l];
        m->u[l] += dt * (m->fx[l] / ms);
        m->v[l] += dt * (m->fy[l] / ms);
        m->w[l] += dt * (m->tq[l] / I);
        m->x[l] -= m->dx * floor(m->x[l] / m->dx);   /* doubly periodic cell */
        m->y[l] -= m->dy * floor(m->y[l] / m->dy);
    }
    /* gradual update towards the coarse solution, Eqs. (3.5-3.7).
     * reading: equal increments n_t/N0 of (target - snapshot) per update step;
     * radius by a uniform scale that hits the coarse mass density. */
    if (ramp) {
        const double *tg = m->tgt;
        int32_t nc = m->ncell;
        double s = tg[c], dvx = tg[nc + c], dvy = tg[2 * nc + c], dw = tg[3 * nc + c];
        for (int64_t l = b; l < e; l++) {
            m->r[l] += (s - 1.0) * m->r0[l] * ramp_frac;
            m->u[l] += dvx * ramp_frac;
            m->v[l] += dvy * ramp_frac;
            m->w[l] += dw * ramp_frac;
        }
    }
    double *mo = m->mom + (size_t)c * ORC_NMOM;
    cell_moments(p, b, e, m->u, m->v, m->w, m->r, m->h, m->fdx, m->fdy, m->tdq, mo);
    if (p->couple) {
        int32_t nc = m->ncell;
        /* data accumulated over the window (Algorithm 1): mass-weighted mean
         * velocity and the cell's total drag */
        if (mo[1] > 0.0) {
            m->win[c] += mo[2] / mo[1];
            m->win[nc + c] += mo[3] / mo[1];
        }
        m->win[2 * nc + c] += mo[9];
        m->win[3 * nc + c] += mo[10];
        m->win[4 * nc + c] += mo[11];
    }
}

/* Coarse step of Algorithm 1 at j = k N0. */
static void model_coarse_step(orc_model *m, double dt)
{
    const orc_params *p = &m->p;
    int32_t nc = m->ncell;
    double Ac = m->dx * m->dy;
    double N0 = (double)p->N0;
    if (!m->have_q) {
        /* initialise the coarse model from the DEM data (Sec. 3.2) */
        for (int32_t c = 0; c < nc; c++) {
            const double *mo = m->mom + (size_t)c * ORC_NMOM;
            m->q[c] = mo[1] / Ac;
            m->q[nc + c] = mo[2] / Ac;
            m->q[2 * nc + c] = mo[3] / Ac;
            m->q[3 * nc + c] = mo[5] / Ac;
        }
        m->have_q = 1;
    }
    double *V = (double *)malloc(sizeof(double) * 2 * nc);
    double *S = (double *)malloc(sizeof(double) * 4 * nc);
    double cmax = 0.0;
    for (int32_t c = 0; c < nc; c++) {
        V[c] = m->win[c] / N0;
        V[nc + c] = m->win[nc + c] / N0;
        S[c] = 0.0;
        S[nc + c] = m->win[2 * nc + c] / N0 / Ac;
        S[2 * nc + c] = m->win[3 * nc + c] / N0 / Ac;
        S[3 * nc + c] = m->win[4 * nc + c] / N0 / Ac;
        double cx = fabs(V[c]) / m->dx, cy = fabs(V[nc + c]) / m->dy;
        double cc = cx > cy ? cx : cy;
        if (cc > cmax) cmax = cc;
    }
    /* CFL (Sec. 3.2): |v| dtau / dX <= 1/2 per direction (reading: the 2-D LF
     * stability limit), so N1 substeps of dtau = dT / N1 */
    double dT = N0 * dt;
    int32_t N1 = (int32_t)ceil(dT * cmax / 0.5);
    if (N1 < 1) N1 = 1;
    orc_lf_bc(p->nx, p->ny, m->dx, m->dy, m->q, V, S, dT / N1, N1, p->walls);
    /* targets of the gradual update over the next coarse step */
    for (int32_t c = 0; c < nc; c++) {
        const double *mo = m->mom + (size_t)c * ORC_NMOM;
        double M = mo[1];
        double s = 1.0, dvx = 0.0, dvy = 0.0, dw = 0.0;
        if (M > 0.0) {
            double rho_dem = M / Ac;
            double qr = m->q[c] > 0.0 ? m->q[c] : 0.0;
            s = sqrt(qr / rho_dem);
            double s2 = s * s, s4 = s2 * s2;
            if (s2 * M > 0.0) {
                dvx = (m->q[nc + c] * Ac - s2 * mo[2]) / (s2 * M);
                dvy = (m->q[2 * nc + c] * Ac - s2 * mo[3]) / (s2 * M);
            }
            if (s4 * mo[4] > 0.0)
                dw = (m->q[3 * nc + c] * Ac - s4 * mo[5]) / (s4 * mo[4]);
        }
        m->tgt[c] = s; m->tgt[nc + c] = dvx; m->tgt[2 * nc + c] = dvy; m->tgt[3 * nc + c] = dw;
    }
    memcpy(m->r0, m->r, sizeof(double) * (m->n > 0 ? m->n : 1));
    memset(m->win, 0, sizeof(double) * ORC_NWIN * nc);
    m->have_tgt = 1;
    free(V);
    free(S);
}

int orc_model_step(orc_model *m, double dt, int64_t nsteps)
{
    const orc_params *p = &m->p;
    if (!(dt > 0.0) || nsteps < 0) return -1;
    if (m->dt == 0.0) m->dt = dt;
    else if (dt != m->dt) return -1;      /* the schedule needs a fixed dt */
    if (p->couple && (p->N0 <= 0 || p->n_t <= 0 || p->N0 % p->n_t != 0)) return -1;
    if (m->coarse_pending) return -1;      /* a held coarse step has to run first */
    for (int64_t k = 0; k < nsteps; k++) {
        int64_t s = m->steps + 1;          /* index of this step, 1-based */
        double t = (double)m->steps * dt;  /* forces at t_n */
        int ramp = p->couple && m->have_tgt && s > p->N0 && (s % p->n_t) == 0;
        double frac = p->couple ? (double)p->n_t / (double)p->N0 : 0.0;
        int32_t nc = m->ncell;
        int32_t c;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(g_threads)
#endif
        for (c = 0; c < nc; c++) model_cell_step(m, c, dt, t, ramp, frac);
        m->steps = s;
        if (p->couple && (s % p->N0) == 0) {
            if (m->hold_coarse) {
                m->coarse_pending = 1;
                return 0;
            }
            model_coarse_step(m, dt);
        }
    }
    return 0;
}

/* Sharded runs (a rank advances the cells it owns and the ranks exchange
 * what the coarse step reads): with hold set, orc_model_step returns right
 * after the last fine step of a coarse interval and leaves the coarse step
 * pending.  The coarse step reads, per cell, the moment columns 1-5 (sum m,
 * sum m u, sum m v, sum I, sum I omega: its initial state and the targets)
 * and the window sums: ORC_NCI values, exported and replaced here. */
void orc_model_set_hold(orc_model *m, int32_t hold) { m->hold_coarse = hold ? 1 : 0; }

void orc_model_coarse_inputs(const orc_model *m, double *out)
{
    int32_t nc = m->ncell;
    for (int32_t c = 0; c < nc; c++) {
        for (int k = 0; k < 5; k++) out[(size_t)c * ORC_NCI + k] = m->mom[(size_t)c * ORC_NMOM + 1 + k];
        for (int k = 0; k < ORC_NWIN; k++) out[(size_t)c * ORC_NCI + 5 + k] = m->win[(size_t)k * nc + c];
    }
}

void orc_model_set_coarse_inputs(orc_model *m, int32_t ncells, const int32_t *cells, const double *vals)
{
    int32_t nc = m->ncell;
    for (int32_t i = 0; i < ncells; i++) {
        int32_t c = cells[i];
        if (c < 0 || c >= nc) continue;
        for (int k = 0; k < 5; k++) m->mom[(size_t)c * ORC_NMOM + 1 + k] = vals[(size_t)i * ORC_NCI + k];
        for (int k = 0; k < ORC_NWIN; k++) m->win[(size_t)k * nc + c] = vals[(size_t)i * ORC_NCI + 5 + k];
    }
}

int32_t orc_model_pending(const orc_model *m) { return m->coarse_pending; }

int orc_model_coarse(orc_model *m)
{
    if (!m->coarse_pending) return -1;
    model_coarse_step(m, m->dt);
    m->coarse_pending = 0;
    return 0;
}

/* Moment columns per cell (Sec. 2.3; drag sums of the last step):
 * 0 n, 1 sum m, 2 sum m u, 3 sum m v, 4 sum I, 5 sum I omega, 6 sum pi r^2,
 * 7 sum m u^2, 8 sum m v^2, 9 sum F_drag,x, 10 sum F_drag,y, 11 sum T_drag */
void orc_model_moments(const orc_model *m, double *out)
{
    memcpy(out, m->mom, sizeof(double) * (size_t)m->ncell * ORC_NMOM);
}

void orc_model_floes(const orc_model *m, double *out)
{
    int64_t n = m->n;
    for (int32_t c = 0; c < m->ncell; c++) {
        int32_t ix = c % m->p.nx, iy = c / m->p.nx;
        for (int64_t k = m->off[c]; k < m->off[c + 1]; k++) {
            int64_t l = m->orig[k];
            out[l] = ix * m->dx + m->x[k];
            out[n + l] = iy * m->dy + m->y[k];
            out[2 * n + l] = m->th[k];
            out[3 * n + l] = m->u[k];
            out[4 * n + l] = m->v[k];
            out[5 * n + l] = m->w[k];
            out[6 * n + l] = m->r[k];
            out[7 * n + l] = m->h[k];
        }
    }
}

void orc_model_coupling(const orc_model *m, double *q, double *targets,
                        double *window, int64_t *flags)
{
    size_t nc = (size_t)m->ncell;
    if (q) memcpy(q, m->q, sizeof(double) * 4 * nc);
    if (targets) memcpy(targets, m->tgt, sizeof(double) * 4 * nc);
    if (window) memcpy(window, m->win, sizeof(double) * ORC_NWIN * nc);
    if (flags) { flags[0] = m->have_q; flags[1] = m->have_tgt; flags[2] = m->steps; }
}

void orc_model_layout(const orc_model *m, int64_t *off, int64_t *orig)
{
    if (off) memcpy(off, m->off, sizeof(int64_t) * (m->ncell + 1));
    if (orig) memcpy(orig, m->orig, sizeof(int64_t) * (m->n > 0 ? m->n : 1));
}

/* ------------------------------------------------------------ truth model */

struct orc_truth {
    orc_params p;
    double *modes;
    int64_t n;
    double *x, *y, *th, *u, *v, *w, *r, *h;
    double *fx, *fy, *tq, *fdx, *fdy, *tdq;
    int64_t steps;
    double dt;
    int brute;                     /* 1: the plain loop over all pairs only */
};

void orc_truth_set_brute(orc_truth *t, int32_t brute) { t->brute = brute ? 1 : 0; }

static int cmp_i64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Contact forces of the truth DEM with a bin search.  Same result, bit for
 * bit, as the loop over all pairs (l < j) in index order: floe l's sums take
 * the pairs (i, l), i < l, in increasing i, then (l, j), j > l, in increasing
 * j, which is the order in which that loop reaches floe l; each pair's force
 * comes from the same orc_pair(lower index, higher index) call, and pairs
 * not in contact add nothing.  Bins of side >= 2 r_max hold every contact
 * partner of a floe within its 3 x 3 neighbourhood.  Returns 0 when the
 * domain is too small for 3 bins per side (the caller uses the plain loop). */
static int truth_forces_binned(orc_truth *t)
{
    const orc_params *p = &t->p;
    const int64_t n = t->n;
    double rmax = 0.0;
    for (int64_t l = 0; l < n; l++) rmax = t->r[l] > rmax ? t->r[l] : rmax;
    if (!(rmax > 0.0)) return 0;
    int64_t nbx = (int64_t)floor(p->Lx / (2.0 * rmax)), nby = (int64_t)floor(p->Ly / (2.0 * rmax));
    if (nbx < 3 || nby < 3) return 0;
    if (nbx > 4096) nbx = 4096;
    if (nby > 4096) nby = 4096;
    const double bx = p->Lx / (double)nbx, by = p->Ly / (double)nby;
    const double Px = p->walls ? 0.0 : p->Lx;     /* no periodic image in x between walls */
    int64_t *start = (int64_t *)calloc((size_t)(nbx * nby + 1), sizeof(int64_t));
    int64_t *bin = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t l = 0; l < n; l++) {
        int64_t ix = (int64_t)floor(t->x[l] / bx), iy = (int64_t)floor(t->y[l] / by);
        ix = ix < 0 ? 0 : (ix >= nbx ? nbx - 1 : ix);
        iy = iy < 0 ? 0 : (iy >= nby ? nby - 1 : iy);
        bin[l] = iy * nbx + ix;
        start[bin[l] + 1]++;
    }
    for (int64_t b = 0; b < nbx * nby; b++) start[b + 1] += start[b];
    {
        int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nbx * nby));
        memcpy(cur, start, sizeof(int64_t) * (size_t)(nbx * nby));
        for (int64_t l = 0; l < n; l++) list[cur[bin[l]]++] = l;   /* ascending within each bin */
        free(cur);
    }
    int64_t l;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 256) num_threads(g_threads)
#endif
    for (l = 0; l < n; l++) {
        int64_t cand[4096];
        int64_t nc = 0;
        const int64_t ix = bin[l] % nbx, iy = bin[l] / nbx;
        int overflow = 0;
        for (int64_t dy = -1; dy <= 1; dy++)
            for (int64_t dx = -1; dx <= 1; dx++) {
                if (p->walls && (ix + dx < 0 || ix + dx >= nbx)) continue;   /* no image across a wall */
                const int64_t jx = (ix + dx + nbx) % nbx, jy = (iy + dy + nby) % nby;
                const int64_t b = jy * nbx + jx;
                for (int64_t k = start[b]; k < start[b + 1]; k++) {
                    if (list[k] == l) continue;
                    if (nc < 4096) cand[nc++] = list[k];
                    else overflow = 1;
                }
            }
        (void)overflow;   /* 4096 partners within 3 x 3 bins cannot occur for disks that do not pile up */
        qsort(cand, (size_t)nc, sizeof(int64_t), cmp_i64);
        double fx = 0.0, fy = 0.0, tq = 0.0, o[16];
        for (int64_t k = 0; k < nc; k++) {
            const int64_t j = cand[k];
            if (j < l) {
                if (orc_pair(p, Px, p->Ly,
                             t->x[j], t->y[j], t->u[j], t->v[j], t->w[j], t->r[j], t->h[j],
                             t->x[l], t->y[l], t->u[l], t->v[l], t->w[l], t->r[l], t->h[l], o)) {
                    fx -= o[0]; fy -= o[1]; tq += o[3];
                }
            } else if (orc_pair(p, Px, p->Ly,
                                t->x[l], t->y[l], t->u[l], t->v[l], t->w[l], t->r[l], t->h[l],
                                t->x[j], t->y[j], t->u[j], t->v[j], t->w[j], t->r[j], t->h[j], o)) {
                fx += o[0]; fy += o[1]; tq += o[2];
            }
        }
        t->fx[l] = fx; t->fy[l] = fy; t->tq[l] = tq;
    }
    free(start);
    free(bin);
    free(list);
    return 1;
}

orc_truth *orc_truth_create(const orc_params *p, int64_t n,
                            const double *x, const double *y, const double *theta,
                            const double *u, const double *v, const double *omega,
                            const double *r, const double *h)
{
    orc_truth *t = (orc_truth *)calloc(1, sizeof(orc_truth));
    copy_params(&t->p, &t->modes, p);
    t->n = n;
    double **arrs[] = {&t->x, &t->y, &t->th, &t->u, &t->v, &t->w, &t->r, &t->h,
                       &t->fx, &t->fy, &t->tq, &t->fdx, &t->fdy, &t->tdq};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); k++)
        *arrs[k] = (double *)calloc(n > 0 ? n : 1, sizeof(double));
    for (int64_t l = 0; l < n; l++) {
        t->x[l] = p->walls ? x[l] : x[l] - p->Lx * floor(x[l] / p->Lx);
        t->y[l] = y[l] - p->Ly * floor(y[l] / p->Ly);
        t->th[l] = theta[l]; t->u[l] = u[l]; t->v[l] = v[l]; t->w[l] = omega[l];
        t->r[l] = r[l]; t->h[l] = h[l];
    }
    return t;
}

void orc_truth_free(orc_truth *t)
{
    if (!t) return;
    double *arrs[] = {t->x, t->y, t->th, t->u, t->v, t->w, t->r, t->h, t->fx, t->fy,
                      t->tq, t->fdx, t->fdy, t->tdq, t->modes};
    for (size_t k = 0; k < sizeof(arrs) / sizeof(arrs[0]); k++) free(arrs[k]);
    free(t);
}

/* The truth: the same DEM (Eq. 2.1) on the whole periodic domain, no
 * localisation and no coupling (Sec. 4); with walls (Sec. 4.4) periodic in y
 * only, and the walls' contact forces added after the floe pairs. */
int orc_truth_step(orc_truth *t, double dt, int64_t nsteps)
{
    const orc_params *p = &t->p;
    if (!(dt > 0.0) || nsteps < 0) return -1;
    if (t->dt == 0.0) t->dt = dt;
    else if (dt != t->dt) return -1;
    int64_t n = t->n;
    double o[16];
    for (int64_t k = 0; k < nsteps; k++) {
        double time = (double)t->steps * dt;
        for (int64_t l = 0; l < n; l++) { t->fx[l] = 0.0; t->fy[l] = 0.0; t->tq[l] = 0.0; }
        const int64_t npl = (!t->brute && truth_forces_binned(t)) ? 0 : n;   /* 0: forces done */
        const double Px = p->walls ? 0.0 : p->Lx;
        for (int64_t l = 0; l < npl; l++)
            for (int64_t j = l + 1; j < n; j++) {
                if (orc_pair(p, Px, p->Ly,
                             t->x[l], t->y[l], t->u[l], t->v[l], t->w[l], t->r[l], t->h[l],
                             t->x[j], t->y[j], t->u[j], t->v[j], t->w[j], t->r[j], t->h[j], o)) {
                    t->fx[l] += o[0]; t->fy[l] += o[1]; t->tq[l] += o[2];
                    t->fx[j] -= o[0]; t->fy[j] -= o[1]; t->tq[j] += o[3];
                }
            }
        if (p->walls)
            for (int64_t l = 0; l < n; l++)
                if (orc_wall(p, p->Lx, t->x[l], t->u[l], t->v[l], t->w[l], t->r[l], t->h[l], o)) {
                    t->fx[l] += o[0]; t->fy[l] += o[1]; t->tq[l] += o[2];
                }
        for (int64_t l = 0; l < n; l++) {
            double f[5], Fx, Fy, T;
            orc_forcing(p, t->x[l], t->y[l], time, f);
            drag(p, f, t->u[l], t->v[l], t->w[l], t->r[l], &Fx, &Fy, &T);
            t->fdx[l] = Fx; t->fdy[l] = Fy; t->tdq[l] = T;
            t->fx[l] += Fx; t->fy[l] += Fy; t->tq[l] += T;
        }
        for (int64_t l = 0; l < n; l++) {
            double ms = floe_mass(p, t->r[l], t->h[l]);
            double I = floe_inertia(p, ms, t->r[l]);
            t->x[l] += dt * t->u[l];
            t->y[l] += dt * t->v[l];
            t->th[l] += dt * t->w[l];
            t->u[l] += dt * (t->fx[l] / ms);
            t->v[l] += dt * (t->fy[l] / ms);
            t->w[l] += dt * (t->tq[l] / I);
            if (!p->walls) t->x[l] -= p->Lx * floor(t->x[l] / p->Lx);
            /* reading: a centre that would pass a wall stays on it */
            else t->x[l] = fmin(fmax(t->x[l], 0.0), p->Lx);
            t->y[l] -= p->Ly * floor(t->y[l] / p->Ly);
        }
        t->steps++;
    }
    return 0;
}

/* Truth floes binned by the coarse cell holding their centre; same columns
 * as orc_model_moments(). */
void orc_truth_moments(const orc_truth *t, double *out)
{
    const orc_params *p = &t->p;
    int32_t nc = p->nx * p->ny;
    double dx = p->Lx / p->nx, dy = p->Ly / p->ny;
    memset(out, 0, sizeof(double) * (size_t)nc * ORC_NMOM);
    for (int64_t l = 0; l < t->n; l++) {
        int32_t ix = cell_index(t->x[l], p->Lx, dx, p->nx);
        int32_t iy = cell_index(t->y[l], p->Ly, dy, p->ny);
        double *mo = out + (size_t)(iy * p->nx + ix) * ORC_NMOM;
        double m = floe_mass(p, t->r[l], t->h[l]);
        double I = floe_inertia(p, m, t->r[l]);
        mo[0] += 1.0;
        mo[1] += m;
        mo[2] += m * t->u[l];
        mo[3] += m * t->v[l];
        mo[4] += I;
        mo[5] += I * t->w[l];
        mo[6] += PI * t->r[l] * t->r[l];
        mo[7] += m * t->u[l] * t->u[l];
        mo[8] += m * t->v[l] * t->v[l];
        mo[9] += t->fdx[l];
        mo[10] += t->fdy[l];
        mo[11] += t->tdq[l];
    }
}

void orc_truth_floes(const orc_truth *t, double *out)
{
    int64_t n = t->n;
    for (int64_t l = 0; l < n; l++) {
        out[l] = t->x[l]; out[n + l] = t->y[l]; out[2 * n + l] = t->th[l];
        out[3 * n + l] = t->u[l]; out[4 * n + l] = t->v[l]; out[5 * n + l] = t->w[l];
        out[6 * n + l] = t->r[l]; out[7 * n + l] = t->h[l];
    }
}

/* ||u||_L2 = sqrt(int u^2), the integral a sum over the coarse cells (Sec. 4.1) */
double orc_l2_diff(int32_t nx, int32_t ny, double dx, double dy,
                   const double *a, const double *b)
{
    double s = 0.0;
    for (int64_t c = 0; c < (int64_t)nx * ny; c++) {
        double e = a[c] - b[c];
        s += e * e * dx * dy;
    }
    return sqrt(s);
}
