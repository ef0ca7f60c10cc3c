/*
 * FP64 CPU oracle of the scattering-graph voxel path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant generator with the CUDA path; it is written
 * to be read against the paper, not to be fast.
 *
 * What it computes (Mikkonen et al., "Scattering graph method for 3D radiative
 * transfer"), in the node-collapsed voxel form:
 *   - Beer-Lambert transmittance of every graph edge from the optical depth
 *     integrated through the extinction grid (Sec. 2, Eq. radiance_effectuality
 *     and the exponential factor of Eq. Fab), by one Amanatides-Woo voxel
 *     traversal per segment;
 *   - the phase-function quadrature weight p' of Eq. F_term_phase on a
 *     Fibonacci lattice (Sec. 3, phase-function integration paragraph) with a
 *     nearest-direction partition of the lattice;
 *   - the scattering coupling C(r, r') of Eq. scatt_coup, used as a
 *     normalised routing weight and, with c_min > 0, to select the edges of
 *     the scattering graph (C > c_min, Sec. 2) with the lattice re-partitioned
 *     among the directions each source keeps;
 *   - the direct solar source S_a (Sec. 2, external source), the linear system
 *     (I - K) x = s of Eq. flux_system (equivalently the series of Eq. fs_sum),
 *     and the final radiance sum toward the instrument (Sec. 2, last equation)
 *     integrated along each line of sight;
 *   - with ORC_ANISO, the edge unknowns of Eq. flux_system: the arrival
 *     direction kept into every scattering (p' of Eq. F_term_phase with the
 *     angle from the incoming edge), summed as the series of Eq. fs_sum.
 * Readings of points the paper leaves open (orientation of F, chain lumping of
 * extinction beyond the stencil, periodic horizontal boundaries, exact tie
 * rules) are the ones listed in the design notes; each is restated at the
 * function that applies it.
 *
 * Pins: every function here is checked by the CPU tests against closed forms,
 * invariants or brute force (DDA exactness, Beer-Lambert slab, discrete single
 * scattering, energy conservation with a black and with a reflecting ground,
 * translation equivariance, dense solve, quadrature sums; the per-cell
 * quadrature weights against integrals over the exact spherical-Voronoi cells:
 * cell areas for q_iso, HG for q_sun, the cosine for q_lamb; for coupling
 * selection, conservation of the re-partitioned sphere and its
 * spherical-Voronoi limit; for the edge form, its reduction to the node form
 * at g = 0 and energy conservation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_MAXDIR 128
#define ORC_MAXGDIR 64

/* slot kinds (the k field of a matrix slot) */
#define ORC_K_SELF 0   /* deposit at the source itself (chain stopped before p1) */
#define ORC_K_GROUND 7 /* chain hit the ground: deposit on a ground column */

/* flags */
#define ORC_SINGLE_SCATTER 1 /* first order only: K and s are zeroed (pin P3) */
#define ORC_NO_SOLVE 2       /* stop after the matrices and the source */
#define ORC_ANISO 4          /* multiple scattering with the arrival direction kept (every order HG) */

typedef struct {
    int nx, ny, nz;
    double hx, hy, hz;
    int R;        /* stencil radius (1 or 2) */
    int M;        /* Fibonacci lattice points */
    int coupling; /* 0: c = 1, 1: normalised coupling weight */
    int S;        /* scattering species */
    double albedo;
    double sza, saa, vza, vaa; /* degrees */
    double f0;
    int npx, npy;
    int flags;
    int threads;
    double gmres_tol;
    int gmres_restart;
    int gmres_maxit;
    double c_min; /* coupling threshold of the scattering graph; 0: full stencil */
    long max_couplings; /* > 0: keep the max_couplings largest couplings (Sec. 3); c_min must be 0 */
} orc_desc;

typedef struct {
    int n_atm, n_ground, n_nodes;
    int n_dirs, n_gdirs;
    int dirs[ORC_MAXDIR * 3];
    int kmax[ORC_MAXDIR];
    int gdir_nmem[ORC_MAXGDIR];
    int gdir_mem[ORC_MAXGDIR * 4 * 3]; /* (dx, dy, dzc) members of each ground chain */
    double q_iso[ORC_MAXDIR];
    double q_lamb[ORC_MAXGDIR];
    double *q_sun; /* [S][n_dirs] */
    double mu_s_lamb;
    double *tsun;  /* [n_nodes] sun transmittance at top-face centre / ground point */
    double *e1;    /* [n_nodes] first-order scattered (reflected) power */
    double *z_iso, *z_sun; /* [n_nodes] coupling normalisers (1 when c = 1) */
    double *esc_iso, *esc_sun; /* [n_nodes] sum_u q c E_{j,u} */
    long n_slots;
    int *slot_row, *slot_col;
    int16_t *slot_dir; /* 0..n_dirs-1 atmospheric, n_dirs + g ground */
    int8_t *slot_k;
    double *slot_dep, *slot_depsun; /* q c P (without the receiver factor) */
    double *slot_val, *slot_valsun; /* rho_row * dep */
    double *s, *x;             /* [n_nodes] */
    double *emis1, *emis_sun, *emis_ms; /* [n_atm] split of E_i */
    double *rad, *refl;        /* [npy][npx] */
    int gmres_iters;
    double rel_resid;
    /* ORC_ANISO only */
    double *slot_P;            /* deposit fraction of each slot (no weights) */
    double *chain_C, *chain_E; /* [n_nodes][n_dirs]: coupling of each chain (-1: no receiver), escape */
    double *X;                 /* [n_nodes][n_dirs + n_gdirs]: scattered power by arrival direction */
    double *arrive, *esc_out;  /* [n_nodes]: power arriving at a node; power its chains carry out of the TOA */
    int aniso_iters;
    /* coupling selection: the threshold applied (0: none), the chains that
     * carry a coupling (have a receiver other than their source) and how
     * many of them were kept */
    double c_min_used;
    long n_couplings, n_kept;
} orc_result;

/* ------------------------------------------------------------------------ */
/* small helpers                                                             */

static int orc_gcd(int a, int b) {
    a = a < 0 ? -a : a;
    b = b < 0 ? -b : b;
    while (b) {
        int t = a % b;
        a = b;
        b = t;
    }
    return a;
}

static int imod(int a, int n) {
    int r = a % n;
    return r < 0 ? r + n : r;
}

/* Henyey-Greenstein phase function, normalised to 1 over the sphere. */
static double orc_hg(double g, double mu) {
    double d = 1.0 + g * g - 2.0 * g * mu;
    return (1.0 - g * g) / (4.0 * ORC_PI * d * sqrt(d));
}

/* ------------------------------------------------------------------------ */
/* Directions.  Atmospheric nodes couple to the voxel centres j + k u for   */
/* primitive lattice vectors u with |u|_inf <= R, k = 1..floor(R/|u|_inf)    */
/* (collinear stencil nodes share one quadrature cell and form a chain: the  */
/* cell of Eq. F_term_phase excludes the exact same direction).  Order:      */
/* dz, then dy, then dx, each ascending from -R.                             */

static void orc_make_dirs(const orc_desc *d, orc_result *r) {
    int R = d->R, n = 0;
    for (int dz = -R; dz <= R; ++dz)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                if (!dx && !dy && !dz) continue;
                if (orc_gcd(orc_gcd(dx, dy), dz) != 1) continue;
                r->dirs[3 * n] = dx;
                r->dirs[3 * n + 1] = dy;
                r->dirs[3 * n + 2] = dz;
                int m = abs(dx);
                if (abs(dy) > m) m = abs(dy);
                if (abs(dz) > m) m = abs(dz);
                r->kmax[n] = R / m;
                ++n;
            }
    r->n_dirs = n;
    /* Ground nodes sit at z = 0 under each column and couple to the voxels
     * (c + (dx, dy), layer dzc - 1), |dx|,|dy| <= R, 1 <= dzc <= R, i.e. along
     * the vector (dx, dy, dzc - 1/2) in cell units.  Collinear members form
     * one chain (one cell); they are detected exactly on the doubled integer
     * vectors (2dx, 2dy, 2dzc - 1). */
    int ng = 0;
    for (int dzc = 1; dzc <= R; ++dzc)
        for (int dy = -R; dy <= R; ++dy)
            for (int dx = -R; dx <= R; ++dx) {
                int a = 2 * dx, b = 2 * dy, c = 2 * dzc - 1;
                int gg = orc_gcd(orc_gcd(a, b), c);
                int pa = a / gg, pb = b / gg, pc = c / gg;
                int found = -1;
                for (int g = 0; g < ng && found < 0; ++g) {
                    int *m0 = &r->gdir_mem[(g * 4) * 3];
                    int a0 = 2 * m0[0], b0 = 2 * m0[1], c0 = 2 * m0[2] - 1;
                    int g0 = orc_gcd(orc_gcd(a0, b0), c0);
                    if (a0 / g0 == pa && b0 / g0 == pb && c0 / g0 == pc) found = g;
                }
                if (found < 0) {
                    found = ng++;
                    r->gdir_nmem[found] = 0;
                }
                int k = r->gdir_nmem[found]++;
                int *mm = &r->gdir_mem[(found * 4 + k) * 3];
                mm[0] = dx;
                mm[1] = dy;
                mm[2] = dzc; /* enumeration is by ascending dzc: chain order */
            }
    r->n_gdirs = ng;
}

/* physical unit vector and length of the cell-unit vector v */
static double orc_unit(const orc_desc *d, const double v[3], double out[3]) {
    double p0 = v[0] * d->hx, p1 = v[1] * d->hy, p2 = v[2] * d->hz;
    double L = sqrt(p0 * p0 + p1 * p1 + p2 * p2);
    out[0] = p0 / L;
    out[1] = p1 / L;
    out[2] = p2 / L;
    return L;
}

static void orc_atm_dir(const orc_desc *d, const orc_result *r, int u, double uhat[3], double *len) {
    double v[3] = {r->dirs[3 * u], r->dirs[3 * u + 1], r->dirs[3 * u + 2]};
    *len = orc_unit(d, v, uhat);
}

static void orc_gnd_dir(const orc_desc *d, const orc_result *r, int g, double uhat[3]) {
    const int *m0 = &r->gdir_mem[(g * 4) * 3];
    double v[3] = {m0[0], m0[1], m0[2] - 0.5};
    orc_unit(d, v, uhat);
}

/* ------------------------------------------------------------------------ */
/* Fibonacci lattice (Gonzalez 2010) and the quadrature weights p' of        */
/* Eq. F_term_phase: each lattice point belongs to the cell of the coupled   */
/* direction closest to it (largest cosine; exact ties to the lowest index), */
/* and a cell's weight is the phase function summed over its points.         */

static void orc_fib_point(int m, int M, double s[3]) {
    const double phi = (1.0 + sqrt(5.0)) / 2.0;
    double z = 1.0 - (2.0 * m + 1.0) / M;
    double q = m / phi;
    double lam = 2.0 * ORC_PI * (q - floor(q));
    double rr = sqrt(1.0 - z * z);
    s[0] = rr * cos(lam);
    s[1] = rr * sin(lam);
    s[2] = z;
}

static void orc_sun_dir(const orc_desc *d, double s0[3]) {
    /* propagation direction of the direct beam (toward the ground) */
    double th = d->sza * ORC_PI / 180.0, ph = d->saa * ORC_PI / 180.0;
    s0[0] = -sin(th) * cos(ph);
    s0[1] = -sin(th) * sin(ph);
    s0[2] = -cos(th);
}

static void orc_view_dir(const orc_desc *d, double v[3]) {
    /* direction from the scene toward the instrument */
    double th = d->vza * ORC_PI / 180.0, ph = d->vaa * ORC_PI / 180.0;
    v[0] = sin(th) * cos(ph);
    v[1] = sin(th) * sin(ph);
    v[2] = cos(th);
}

static void orc_quadrature(const orc_desc *d, const double *g, orc_result *r) {
    int M = d->M, nd = r->n_dirs, ng = r->n_gdirs, S = d->S;
    double uh[ORC_MAXDIR][3], gh[ORC_MAXGDIR][3], len;
    for (int u = 0; u < nd; ++u) orc_atm_dir(d, r, u, uh[u], &len);
    for (int k = 0; k < ng; ++k) orc_gnd_dir(d, r, k, gh[k]);
    double s0[3];
    orc_sun_dir(d, s0);
    long cnt[ORC_MAXDIR];
    double zsum[ORC_MAXGDIR], ztot = 0.0;
    memset(cnt, 0, sizeof cnt);
    memset(zsum, 0, sizeof zsum);
    double *hsum = calloc((size_t)S * nd, sizeof(double));
    double *htot = calloc((size_t)S, sizeof(double));
    for (int m = 0; m < M; ++m) {
        double sm[3];
        orc_fib_point(m, M, sm);
        int best = 0;
        double bc = uh[0][0] * sm[0] + uh[0][1] * sm[1] + uh[0][2] * sm[2];
        for (int u = 1; u < nd; ++u) {
            double c = uh[u][0] * sm[0] + uh[u][1] * sm[1] + uh[u][2] * sm[2];
            if (c > bc) {
                bc = c;
                best = u;
            }
        }
        cnt[best]++;
        double mu0 = s0[0] * sm[0] + s0[1] * sm[1] + s0[2] * sm[2];
        for (int sp = 0; sp < S; ++sp) {
            double h = orc_hg(g[sp], mu0);
            hsum[sp * nd + best] += h;
            htot[sp] += h;
        }
        if (sm[2] > 0.0) {
            int gb = 0;
            double gc = gh[0][0] * sm[0] + gh[0][1] * sm[1] + gh[0][2] * sm[2];
            for (int k = 1; k < ng; ++k) {
                double c = gh[k][0] * sm[0] + gh[k][1] * sm[1] + gh[k][2] * sm[2];
                if (c > gc) {
                    gc = c;
                    gb = k;
                }
            }
            zsum[gb] += sm[2];
            ztot += sm[2];
        }
    }
    for (int u = 0; u < nd; ++u) r->q_iso[u] = (double)cnt[u] / (double)M;
    for (int k = 0; k < ng; ++k) r->q_lamb[k] = zsum[k] / ztot;
    for (int sp = 0; sp < S; ++sp)
        for (int u = 0; u < nd; ++u) r->q_sun[sp * nd + u] = hsum[sp * nd + u] / htot[sp];
    free(hsum);
    free(htot);
}

/* ------------------------------------------------------------------------ */
/* Optical depth by voxel traversal (Amanatides & Woo 1987).                 */
/* The ray starts at P (cell units: x/hx, y/hy, z/hz), moves by V cell units */
/* per unit parameter t, for t in [0, tend]; lphys is the physical length    */
/* per unit t.  x and y are periodic; z is bounded by the ground and the TOA.*/
/* A start exactly on a cell face belongs to the cell the ray enters.  A     */
/* simultaneous crossing of several faces steps one axis at a time, so the   */
/* cells passed at a corner get a zero-length piece, which adds nothing.     */
/* If segs is not NULL, each traversed piece is reported as (cell, t0, t1).  */

typedef void (*orc_seg_fn)(void *ctx, int cell, double t0, double t1);

double orc_dda(const orc_desc *d, const double *mu_e, const double P[3], const double V[3], double tend,
               double lphys, orc_seg_fn fn, void *ctx) {
    int c[3], step[3];
    double tnext[3], tau = 0.0;
    const int n[3] = {d->nx, d->ny, d->nz};
    for (int a = 0; a < 3; ++a) {
        if (V[a] > 0.0) {
            c[a] = (int)floor(P[a]);
            step[a] = 1;
            tnext[a] = ((double)(c[a] + 1) - P[a]) / V[a];
        } else if (V[a] < 0.0) {
            c[a] = (int)ceil(P[a]) - 1;
            step[a] = -1;
            tnext[a] = ((double)c[a] - P[a]) / V[a];
        } else {
            c[a] = (int)floor(P[a]);
            step[a] = 0;
            tnext[a] = INFINITY;
        }
    }
    double t = 0.0;
    while (t < tend) {
        int a = 0;
        if (tnext[1] < tnext[a]) a = 1;
        if (tnext[2] < tnext[a]) a = 2;
        double t1 = tnext[a] < tend ? tnext[a] : tend;
        if (t1 > t) {
            if (c[2] < 0 || c[2] >= n[2]) {
                /* only reachable through rounding at the very end of a ray */
            } else {
                int cell = (c[2] * n[1] + imod(c[1], n[1])) * n[0] + imod(c[0], n[0]);
                tau += mu_e[cell] * (t1 - t) * lphys;
                if (fn) fn(ctx, cell, t, t1);
            }
        }
        t = t1;
        if (t >= tend) break;
        c[a] += step[a];
        tnext[a] = ((double)(step[a] > 0 ? c[a] + 1 : c[a]) - P[a]) / V[a];
    }
    return tau;
}

/* ------------------------------------------------------------------------ */
/* Chain march for one source and one direction (deposit fractions).         */
/* Reading of the lumping: the chain p0 = r_j, p1, ... p_m stops when the    */
/* stencil ends inside the domain (a), or the ray leaves through the TOA (b) */
/* or the ground (c) before p_{m+1}.  Node p_k gets T_{k-1}(1 - e^{-tau_k}); */
/* the terminal node (or the source when m = 0) also gets T_m(1 - T_beyond), */
/* T_beyond being the transmittance to the TOA for upward travel in (a) and  */
/* (b), the transmittance to the ground hit in (c), and 0 for horizontal or  */
/* downward travel in (a).  Ground columns get T_m T_hit in (c).  Escape is  */
/* T_m T_TOA for upward travel, 0 otherwise.  The fractions sum to 1.        */

typedef struct {
    int node;    /* receiver node id */
    int k;       /* chain index, ORC_K_SELF or ORC_K_GROUND */
    double P;    /* deposit fraction */
} orc_dep;

typedef struct {
    int ndep;
    orc_dep dep[16];
    double escape;
    int first;        /* first receiver other than the source, -1 if none */
    double first_dist;/* physical distance to it (to the hit point for ground) */
} orc_chain;

static int atm_node(const orc_desc *d, int ix, int iy, int iz) {
    return (iz * d->ny + imod(iy, d->ny)) * d->nx + imod(ix, d->nx);
}

static void chain_add(orc_chain *ch, int node, int k, double P) {
    for (int i = 0; i < ch->ndep; ++i)
        if (ch->dep[i].node == node && ch->dep[i].k == k) {
            ch->dep[i].P += P;
            return;
        }
    ch->dep[ch->ndep].node = node;
    ch->dep[ch->ndep].k = k;
    ch->dep[ch->ndep].P = P;
    ch->ndep++;
}

static void orc_atm_chain(const orc_desc *d, const orc_result *r, const double *mu_e, int j, int u,
                          orc_chain *ch) {
    int nx = d->nx, ny = d->ny, nz = d->nz, nxy = nx * ny;
    int iz = j / nxy, iy = (j / nx) % ny, ix = j % nx;
    const int *v = &r->dirs[3 * u];
    double V[3] = {v[0], v[1], v[2]};
    double uh[3], L;
    orc_atm_dir(d, r, u, uh, &L);
    double P[3] = {ix + 0.5, iy + 0.5, iz + 0.5};
    int cx = ix, cy = iy, cz = iz, prev = j;
    double tau_pre = 0.0;
    ch->ndep = 0;
    ch->escape = 0.0;
    ch->first = -1;
    ch->first_dist = 0.0;
    int k;
    for (k = 1; k <= r->kmax[u]; ++k) {
        double znext = P[2] + V[2];
        if (znext > nz) { /* (b) leaves through the TOA before p_k */
            double tb = ((double)nz - P[2]) / V[2];
            double taub = orc_dda(d, mu_e, P, V, tb, L, NULL, NULL);
            chain_add(ch, prev, k == 1 ? ORC_K_SELF : k - 1, exp(-tau_pre) * (-expm1(-taub)));
            ch->escape = exp(-(tau_pre + taub));
            return;
        }
        if (znext < 0.0) { /* (c) hits the ground before p_k */
            double th = P[2] / -V[2];
            double tauc = orc_dda(d, mu_e, P, V, th, L, NULL, NULL);
            chain_add(ch, prev, k == 1 ? ORC_K_SELF : k - 1, exp(-tau_pre) * (-expm1(-tauc)));
            double Tg = exp(-(tau_pre + tauc));
            /* hit point; exact in cell units for R <= 2 (quarter cells) */
            double hx_ = P[0] + th * V[0], hy_ = P[1] + th * V[1];
            int xs[2], ys[2], nxs = 1, nys = 1;
            if (hx_ == floor(hx_)) {
                xs[0] = (int)hx_ - 1;
                xs[1] = (int)hx_;
                nxs = 2;
            } else
                xs[0] = (int)floor(hx_);
            if (hy_ == floor(hy_)) {
                ys[0] = (int)hy_ - 1;
                ys[1] = (int)hy_;
                nys = 2;
            } else
                ys[0] = (int)floor(hy_);
            double w = 1.0 / (nxs * nys);
            for (int a = 0; a < nxs; ++a)
                for (int b = 0; b < nys; ++b) {
                    int gnode = d->nx * d->ny * d->nz + imod(ys[b], ny) * nx + imod(xs[a], nx);
                    chain_add(ch, gnode, ORC_K_GROUND, Tg * w);
                }
            if (k == 1) {
                ch->first = nxy * nz; /* any ground node: all share mu_s^Lamb */
                ch->first_dist = th * L;
            }
            ch->escape = 0.0;
            return;
        }
        double taus = orc_dda(d, mu_e, P, V, 1.0, L, NULL, NULL);
        cx += v[0];
        cy += v[1];
        cz += v[2];
        P[0] += V[0];
        P[1] += V[1];
        P[2] += V[2];
        int node = atm_node(d, cx, cy, cz);
        chain_add(ch, node, k, exp(-tau_pre) * (-expm1(-taus)));
        if (k == 1) {
            ch->first = node;
            ch->first_dist = L;
        }
        tau_pre += taus;
        prev = node;
    }
    /* (a) the stencil ended inside the domain at p_m = prev */
    int m = k - 1;
    if (V[2] > 0.0) {
        double tb = ((double)nz - P[2]) / V[2];
        double tinf = orc_dda(d, mu_e, P, V, tb, L, NULL, NULL);
        chain_add(ch, prev, m, exp(-tau_pre) * (-expm1(-tinf)));
        ch->escape = exp(-(tau_pre + tinf));
    } else {
        chain_add(ch, prev, m, exp(-tau_pre));
        ch->escape = 0.0;
    }
}

static void orc_gnd_chain(const orc_desc *d, const orc_result *r, const double *mu_e, int c, int g,
                          orc_chain *ch) {
    int nx = d->nx, ny = d->ny, nz = d->nz;
    int ix = c % nx, iy = c / nx;
    double P[3] = {ix + 0.5, iy + 0.5, 0.0};
    double tau_pre = 0.0;
    int prev = d->nx * d->ny * d->nz + c;
    ch->ndep = 0;
    ch->escape = 0.0;
    ch->first = -1;
    ch->first_dist = 0.0;
    int nm = r->gdir_nmem[g];
    int k;
    for (k = 1; k <= nm; ++k) {
        const int *mm = &r->gdir_mem[(g * 4 + k - 1) * 3];
        double Q[3] = {ix + 0.5 + mm[0], iy + 0.5 + mm[1], mm[2] - 0.5};
        double V[3] = {Q[0] - P[0], Q[1] - P[1], Q[2] - P[2]};
        double uh[3];
        double L = orc_unit(d, V, uh);
        if (Q[2] > nz) { /* (b) */
            double tb = ((double)nz - P[2]) / V[2];
            double taub = orc_dda(d, mu_e, P, V, tb, L, NULL, NULL);
            chain_add(ch, prev, k == 1 ? ORC_K_SELF : k - 1, exp(-tau_pre) * (-expm1(-taub)));
            ch->escape = exp(-(tau_pre + taub));
            return;
        }
        double taus = orc_dda(d, mu_e, P, V, 1.0, L, NULL, NULL);
        int node = atm_node(d, ix + mm[0], iy + mm[1], mm[2] - 1);
        chain_add(ch, node, k, exp(-tau_pre) * (-expm1(-taus)));
        if (k == 1) {
            ch->first = node;
            ch->first_dist = L;
        }
        tau_pre += taus;
        prev = node;
        P[0] = Q[0];
        P[1] = Q[1];
        P[2] = Q[2];
    }
    /* (a) the chain ended inside the domain: escape to the TOA along the
     * ground direction from the terminal node */
    int m = k - 1;
    const int *m0 = &r->gdir_mem[(g * 4) * 3];
    double V[3] = {m0[0], m0[1], m0[2] - 0.5};
    double uh[3];
    double L = orc_unit(d, V, uh);
    double tb = ((double)nz - P[2]) / V[2];
    double tinf = orc_dda(d, mu_e, P, V, tb, L, NULL, NULL);
    chain_add(ch, prev, m, exp(-tau_pre) * (-expm1(-tinf)));
    ch->escape = exp(-(tau_pre + tinf));
}

/* ------------------------------------------------------------------------ */
/* Matrices K and K^sun (rows = receivers, reading K = F^T of Eq. Fab), the   */
/* direct source, and the split of every deposit by quadrature weight and    */
/* coupling.                                                                 */
/*   q: p' of Eq. F_term_phase as a probability (isotropic cell fraction for */
/*      orders >= 2, HG-weighted cell fraction for the direct beam, cosine-  */
/*      weighted for the Lambertian ground).                                 */
/*   c: C(r, r') of Eq. scatt_coup between the source and the chain's first  */
/*      receiver, normalised so that sum_u q c = 1 over the directions that  */
/*      have a receiver other than the source (c = 1 elsewhere).             */

/* Scattering coupling of Eq. scatt_coup between a source and the first
 * receiver of its chain along one direction: sqrt(mu_s mu_s') / distance,
 * with mu_s^Lamb for a ground receiver; -1 for a chain without a receiver. */
static double orc_coupling(const orc_result *r, const double *mu_s_tot, const orc_chain *ch, double mus_src) {
    if (ch->first < 0) return -1.0;
    double mus_n = ch->first >= r->n_atm ? r->mu_s_lamb : mu_s_tot[ch->first];
    return sqrt(mus_src * mus_n) / ch->first_dist;
}

/* Quadrature weights of one source over the directions it keeps (coupling
 * selection, Sec. 2: the scattering graph holds the edges with C > c_min).
 * The cells of Eq. F_term_phase are re-drawn among the kept directions: every
 * lattice point joins the kept direction closest to it (largest cosine, exact
 * ties to the lowest index), which is where the flood fill of Sec. 3 over the
 * lattice adjacency, seeded at the kept directions, ends up.  Atmospheric
 * source: qi[u] = points / M and qsun[sp][u] = the HG weight toward the
 * cell over the whole-sphere total; ground source: qi[k] = the cosine-
 * weighted share of the upper hemisphere (qsun unused).  With every
 * direction kept this repeats orc_quadrature's sums in the same order.  A
 * source that keeps nothing gets zero weights. */
static void orc_partition_kept(const orc_desc *d, const orc_result *r, const double *g, int ground, const int *kept,
                               double *qi, double *qsun) {
    int M = d->M, S = d->S;
    int n = ground ? r->n_gdirs : r->n_dirs;
    double uh[ORC_MAXDIR][3], len;
    for (int u = 0; u < n; ++u) {
        if (ground)
            orc_gnd_dir(d, r, u, uh[u]);
        else
            orc_atm_dir(d, r, u, uh[u], &len);
    }
    double s0[3];
    orc_sun_dir(d, s0);
    long cnt[ORC_MAXDIR];
    double zsum[ORC_MAXGDIR], ztot = 0.0;
    memset(cnt, 0, sizeof cnt);
    memset(zsum, 0, sizeof zsum);
    double *hsum = calloc((size_t)S * n, sizeof(double));
    double *htot = calloc((size_t)S, sizeof(double));
    for (int m = 0; m < M; ++m) {
        double sm[3];
        orc_fib_point(m, M, sm);
        if (ground && !(sm[2] > 0.0)) continue;
        int best = -1;
        double bc = 0.0;
        for (int u = 0; u < n; ++u) {
            if (!kept[u]) continue;
            double c = uh[u][0] * sm[0] + uh[u][1] * sm[1] + uh[u][2] * sm[2];
            if (best < 0 || c > bc) {
                bc = c;
                best = u;
            }
        }
        if (ground) {
            if (best >= 0) zsum[best] += sm[2];
            ztot += sm[2];
            continue;
        }
        if (best >= 0) cnt[best]++;
        double mu0 = s0[0] * sm[0] + s0[1] * sm[1] + s0[2] * sm[2];
        for (int sp = 0; sp < S; ++sp) {
            double h = orc_hg(g[sp], mu0);
            if (best >= 0) hsum[sp * n + best] += h;
            htot[sp] += h;
        }
    }
    if (ground) {
        for (int k = 0; k < n; ++k) qi[k] = zsum[k] / ztot;
    } else {
        for (int u = 0; u < n; ++u) qi[u] = (double)cnt[u] / (double)M;
        for (int sp = 0; sp < S; ++sp)
            for (int u = 0; u < n; ++u) qsun[sp * n + u] = hsum[sp * n + u] / htot[sp];
    }
    free(hsum);
    free(htot);
}

/* Which directions a source keeps: those whose chain has a receiver with
 * C > c_min, and every chain without a receiver (it carries no coupling).
 * c_min = 0 keeps the full stencil.  Returns the number dropped. */
static int orc_select(const orc_desc *d, const orc_result *r, const double *mu_s_tot, const orc_chain *ch, int ndir,
                      double mus_src, int *kept) {
    int ndrop = 0;
    for (int u = 0; u < ndir; ++u) {
        double C = orc_coupling(r, mu_s_tot, &ch[u], mus_src);
        kept[u] = !(d->c_min > 0.0) || C < 0.0 || C > d->c_min;
        ndrop += !kept[u];
    }
    return ndrop;
}

/* Routing weight of G15: c_u = C_u sum_v q_v / sum_v q_v C_v over the
 * directions with a receiver (C_v >= 0), 1 for a direction without one; 1
 * everywhere when the coupling is off or the weighted sum is 0.  *zout gets
 * sum q C / sum q (1 in those cases). */
static void orc_route(const orc_desc *d, const double *C, const double *qdir, int ndir, double *cw, double *zout) {
    double sq = 0.0, sqc = 0.0;
    for (int u = 0; u < ndir; ++u) {
        if (C[u] < 0.0) continue;
        sq += qdir[u];
        sqc += qdir[u] * C[u];
    }
    if (d->coupling == 0 || !(sqc > 0.0)) {
        for (int u = 0; u < ndir; ++u) cw[u] = 1.0;
        *zout = 1.0;
        return;
    }
    for (int u = 0; u < ndir; ++u) cw[u] = C[u] >= 0.0 ? C[u] * sq / sqc : 1.0;
    *zout = sqc / sq;
}

static void orc_source_weights(const orc_desc *d, const orc_result *r, const double *mu_s_tot,
                               const double *qdir, int ndir, const orc_chain *ch, int src_is_ground,
                               double mus_src, double *cw, double *zout) {
    /* qdir: q_{j,u}; returns c_{j,u} in cw */
    double C[ORC_MAXDIR];
    (void)src_is_ground;
    for (int u = 0; u < ndir; ++u) C[u] = orc_coupling(r, mu_s_tot, &ch[u], mus_src);
    orc_route(d, C, qdir, ndir, cw, zout);
}

static void orc_ray_sun(const orc_desc *d, const double *mu_e, const double P[3], double *T) {
    double s0[3];
    orc_sun_dir(d, s0);
    double V[3] = {-s0[0] / d->hx, -s0[1] / d->hy, -s0[2] / d->hz};
    double tend = ((double)d->nz - P[2]) * d->hz / -s0[2];
    *T = exp(-orc_dda(d, mu_e, P, V, tend, 1.0, NULL, NULL));
}

/* ------------------------------------------------------------------------ */
/* Solver: restarted GMRES with modified Gram-Schmidt on (I - K) x = s.      */

static void spmv_ImK(const orc_result *r, const int *rowptr, const int *col, const double *val, const double *x,
                     double *y) {
    int n = r->n_nodes;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) acc += val[e] * x[col[e]];
        y[i] = x[i] - acc;
    }
}

static double dotv(const double *a, const double *b, int n) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void orc_gmres(const orc_desc *d, orc_result *r, const int *rowptr, const int *col, const double *val) {
    int n = r->n_nodes, m = d->gmres_restart > 0 ? d->gmres_restart : 60;
    double tol = d->gmres_tol > 0 ? d->gmres_tol : 1e-13;
    int maxit = d->gmres_maxit > 0 ? d->gmres_maxit : 5000;
    double *V = malloc(sizeof(double) * (size_t)n * (m + 1));
    double *H = calloc((size_t)(m + 1) * m, sizeof(double));
    double *cs = malloc(sizeof(double) * m), *sn = malloc(sizeof(double) * m), *gv = malloc(sizeof(double) * (m + 1));
    double *w = malloc(sizeof(double) * n), *rr = malloc(sizeof(double) * n);
    double bn = sqrt(dotv(r->s, r->s, n));
    int it = 0;
    memset(r->x, 0, sizeof(double) * n);
    if (bn == 0.0) {
        r->gmres_iters = 0;
        r->rel_resid = 0.0;
        goto done;
    }
    for (;;) {
        spmv_ImK(r, rowptr, col, val, r->x, w);
        for (int i = 0; i < n; ++i) rr[i] = r->s[i] - w[i];
        double beta = sqrt(dotv(rr, rr, n));
        r->rel_resid = beta / bn;
        if (beta / bn <= tol || it >= maxit) break;
        for (int i = 0; i < n; ++i) V[i] = rr[i] / beta;
        memset(gv, 0, sizeof(double) * (m + 1));
        gv[0] = beta;
        int kk;
        for (kk = 0; kk < m; ++kk) {
            ++it;
            spmv_ImK(r, rowptr, col, val, &V[(size_t)kk * n], w);
            for (int jj = 0; jj <= kk; ++jj) {
                double h = dotv(w, &V[(size_t)jj * n], n);
                H[jj * m + kk] = h;
                for (int i = 0; i < n; ++i) w[i] -= h * V[(size_t)jj * n + i];
            }
            double hn = sqrt(dotv(w, w, n));
            H[(kk + 1) * m + kk] = hn;
            if (hn > 0.0)
                for (int i = 0; i < n; ++i) V[(size_t)(kk + 1) * n + i] = w[i] / hn;
            for (int jj = 0; jj < kk; ++jj) {
                double a = H[jj * m + kk], b = H[(jj + 1) * m + kk];
                H[jj * m + kk] = cs[jj] * a + sn[jj] * b;
                H[(jj + 1) * m + kk] = -sn[jj] * a + cs[jj] * b;
            }
            double a = H[kk * m + kk], b = H[(kk + 1) * m + kk];
            double den = sqrt(a * a + b * b);
            cs[kk] = den > 0 ? a / den : 1.0;
            sn[kk] = den > 0 ? b / den : 0.0;
            H[kk * m + kk] = den;
            H[(kk + 1) * m + kk] = 0.0;
            gv[kk + 1] = -sn[kk] * gv[kk];
            gv[kk] = cs[kk] * gv[kk];
            if (fabs(gv[kk + 1]) / bn <= 0.1 * tol || hn == 0.0 || it >= maxit) {
                ++kk;
                break;
            }
        }
        if (kk > m) kk = m;
        /* back substitution and update */
        double *y = malloc(sizeof(double) * kk);
        for (int i = kk - 1; i >= 0; --i) {
            double acc = gv[i];
            for (int jj = i + 1; jj < kk; ++jj) acc -= H[i * m + jj] * y[jj];
            y[i] = acc / H[i * m + i];
        }
        for (int jj = 0; jj < kk; ++jj)
            for (int i = 0; i < n; ++i) r->x[i] += y[jj] * V[(size_t)jj * n + i];
        free(y);
    }
    r->gmres_iters = it;
done:
    free(V);
    free(H);
    free(cs);
    free(sn);
    free(gv);
    free(w);
    free(rr);
}

/* ------------------------------------------------------------------------ */
/* Detector: line of sight of pixel (a, b) meets the ground at the pixel     */
/* centre and runs along v to the TOA.  Walking from the TOA down, each      */
/* voxel adds e^{-tau_in} f E_i / V with f = (1 - e^{-mu_e ds}) / mu_e, the  */
/* ground adds e^{-tau_tot} (e1_c + x_c) / (pi hx hy).  This integrates the  */
/* final radiance sum of Sec. 2 over voxel segments.                         */

typedef struct {
    const double *mu_e;
    const double *emis; /* E_i */
    double vol, lphys;
    double tau, L;
} orc_los;

static void los_seg(void *ctx, int cell, double t0, double t1) {
    orc_los *c = ctx;
    double ds = (t1 - t0) * c->lphys;
    double me = c->mu_e[cell];
    double f = me > 0.0 ? -expm1(-me * ds) / me : ds;
    c->L += exp(-c->tau) * f * c->emis[cell] / c->vol;
    c->tau += me * ds;
}

/* ------------------------------------------------------------------------ */

void orc_free(orc_result *r);

/* ------------------------------------------------------------------------ */
/* Anisotropic multiple scattering: the edge unknowns of Eq. flux_system.    */
/* phi per directed edge carries its arrival direction into the next         */
/* scattering; the edges that reach a node along one direction are merged    */
/* (re-emission there depends on the arrival direction only), so the unknown */
/* is the power scattered at node i from light that arrived along w, X(i,w). */

/* p' of Eq. F_term_phase with the arrival direction kept: for every arrival
 * direction w (the atmospheric directions, then the ground chains' upward
 * directions) and species, the HG weight toward each lattice point, the angle
 * measured from w, summed over the cell of each atmospheric direction (the
 * nearest-direction partition of orc_quadrature) and divided by the
 * whole-sphere sum: Q[sp][w][u], every row summing to one. */
static void orc_phase_quadrature_fill(const orc_desc *d, const orc_result *r, const double *g, double *Q) {
    int M = d->M, nd = r->n_dirs, ngd = r->n_gdirs, S = d->S, nin = nd + ngd;
    double uh[ORC_MAXDIR][3], wh[ORC_MAXDIR + ORC_MAXGDIR][3], len;
    for (int u = 0; u < nd; ++u) {
        orc_atm_dir(d, r, u, uh[u], &len);
        memcpy(wh[u], uh[u], sizeof uh[u]);
    }
    for (int k = 0; k < ngd; ++k) orc_gnd_dir(d, r, k, wh[nd + k]);
    int *cell = malloc(sizeof(int) * M);
    double *pt = malloc(sizeof(double) * 3 * (size_t)M);
    for (int m = 0; m < M; ++m) {
        double *sm = pt + 3 * (size_t)m;
        orc_fib_point(m, M, sm);
        int best = 0;
        double bc = uh[0][0] * sm[0] + uh[0][1] * sm[1] + uh[0][2] * sm[2];
        for (int u = 1; u < nd; ++u) {
            double c = uh[u][0] * sm[0] + uh[u][1] * sm[1] + uh[u][2] * sm[2];
            if (c > bc) {
                bc = c;
                best = u;
            }
        }
        cell[m] = best;
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int w = 0; w < nin; ++w)
        for (int sp = 0; sp < S; ++sp) {
            double *row = Q + ((size_t)sp * nin + w) * nd;
            double tot = 0.0;
            for (int u = 0; u < nd; ++u) row[u] = 0.0;
            for (int m = 0; m < M; ++m) {
                const double *sm = pt + 3 * (size_t)m;
                double h = orc_hg(g[sp], wh[w][0] * sm[0] + wh[w][1] * sm[1] + wh[w][2] * sm[2]);
                row[cell[m]] += h;
                tot += h;
            }
            for (int u = 0; u < nd; ++u) row[u] /= tot;
        }
    free(cell);
    free(pt);
}

/* The series of Eq. fs_sum over the edge unknowns, phi = S + F S + F^2 S ...,
 * in the merged form:
 *   L(j,u)  = sum_w X(j,w) Q_j(w -> u) c_j(u | w)   power leaving atmospheric j along u
 *             (Q_j: species mixture of Q by the source's mu_s shares; c: the
 *             routing weight of G15 normalised with Q_j(w -> .))
 *   L(c,k)  = (sum_w X(c,w)) q_lamb_k c_k           Lambertian node: no memory of w
 *   X(i,w)  = Xs(i,w) + rho_i sum_{chains (j,u=w) depositing on i} P L(j,u)
 * with Xs the first-order part (the sun's light scattered once at j and
 * arriving at i), iterated until the relative change is below 1e-15.
 * Fills r->X, r->x (the total, as the isotropic solve does), r->arrive and
 * r->esc_out.  Returns 0, or 3 when the weights do not fit in memory. */
static int orc_aniso(const orc_desc *d, orc_result *r, const double *g, const double *mu_s, const double *mus,
                     const double *om, const int *rowcnt) {
    int na = r->n_atm, nn = r->n_nodes, nd = r->n_dirs, ngd = r->n_gdirs, S = d->S, nin = nd + ngd;
    int ng = nn - na;
    double *Q = malloc(sizeof(double) * (size_t)S * nin * nd);
    double *W = malloc(sizeof(double) * (size_t)na * nin * nd);
    if (!Q || !W) {
        free(Q);
        free(W);
        return 3;
    }
    orc_phase_quadrature_fill(d, r, g, Q);
#pragma omp parallel for schedule(static)
    for (int j = 0; j < na; ++j) {
        double q[ORC_MAXDIR], cw[ORC_MAXDIR], z, wsp[16];
        for (int sp = 0; sp < S; ++sp) wsp[sp] = mus[j] > 0.0 ? mu_s[(size_t)sp * na + j] / mus[j] : 1.0 / S;
        for (int w = 0; w < nin; ++w) {
            for (int u = 0; u < nd; ++u) {
                double acc = 0.0;
                for (int sp = 0; sp < S; ++sp) acc += wsp[sp] * Q[((size_t)sp * nin + w) * nd + u];
                q[u] = acc;
            }
            orc_route(d, &r->chain_C[(size_t)j * nd], q, nd, cw, &z);
            for (int u = 0; u < nd; ++u) W[((size_t)j * nin + w) * nd + u] = q[u] * cw[u];
        }
    }
    double *Wg = malloc(sizeof(double) * (size_t)(ng > 0 ? ng : 1) * (ngd > 0 ? ngd : 1));
    for (int c = 0; c < ng; ++c) {
        double cw[ORC_MAXGDIR], z;
        orc_route(d, &r->chain_C[(size_t)(na + c) * nd], r->q_lamb, ngd, cw, &z);
        for (int k = 0; k < ngd; ++k) Wg[(size_t)c * ngd + k] = r->q_lamb[k] * cw[k];
    }
    size_t nx = (size_t)nn * nin;
    double *Xs = calloc(nx, sizeof(double)), *X = calloc(nx, sizeof(double)), *Arr = calloc(nx, sizeof(double));
    double *L = calloc((size_t)nn * nd, sizeof(double));
    double *first = calloc(nn, sizeof(double));
    for (int i = 0; i < nn; ++i) {
        double rho = i < na ? om[i] : d->albedo;
        for (int e = rowcnt[i]; e < rowcnt[i + 1]; ++e) {
            double a = r->slot_depsun[e] * r->e1[r->slot_col[e]];
            Xs[(size_t)i * nin + r->slot_dir[e]] += rho * a;
            first[i] += a;
        }
    }
    memcpy(X, Xs, sizeof(double) * nx);
    int it;
    for (it = 0; it < 100000; ++it) {
#pragma omp parallel for schedule(static)
        for (int j = 0; j < nn; ++j) {
            if (j < na) {
                for (int u = 0; u < nd; ++u) {
                    double acc = 0.0;
                    for (int w = 0; w < nin; ++w) acc += X[(size_t)j * nin + w] * W[((size_t)j * nin + w) * nd + u];
                    L[(size_t)j * nd + u] = acc;
                }
            } else {
                double xt = 0.0;
                for (int w = 0; w < nin; ++w) xt += X[(size_t)j * nin + w];
                for (int k = 0; k < ngd; ++k) L[(size_t)j * nd + k] = xt * Wg[(size_t)(j - na) * ngd + k];
            }
        }
        double num = 0.0, den = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : num, den)
        for (int i = 0; i < nn; ++i) {
            double *ar = Arr + (size_t)i * nin;
            for (int w = 0; w < nin; ++w) ar[w] = 0.0;
            for (int e = rowcnt[i]; e < rowcnt[i + 1]; ++e) {
                int src = r->slot_col[e], dir = r->slot_dir[e];
                int loc = dir < nd ? dir : dir - nd;
                ar[dir] += L[(size_t)src * nd + loc] * r->slot_P[e];
            }
            double rho = i < na ? om[i] : d->albedo;
            for (int w = 0; w < nin; ++w) {
                size_t q = (size_t)i * nin + w;
                double xn = Xs[q] + rho * ar[w];
                num += (xn - X[q]) * (xn - X[q]);
                den += xn * xn;
                X[q] = xn;
            }
        }
        if (num <= 1e-30 * den) break;
    }
    r->aniso_iters = it + 1;
    r->X = X;
    r->arrive = calloc(nn, sizeof(double));
    r->esc_out = calloc(nn, sizeof(double));
    for (int i = 0; i < nn; ++i) {
        double xt = 0.0, at = first[i];
        for (int w = 0; w < nin; ++w) {
            xt += X[(size_t)i * nin + w];
            at += Arr[(size_t)i * nin + w];
        }
        r->x[i] = xt;
        r->arrive[i] = at;
        int n = i < na ? nd : ngd;
        double eo = r->e1[i] * r->esc_sun[i];
        for (int u = 0; u < n; ++u) eo += L[(size_t)i * nd + u] * r->chain_E[(size_t)i * nd + u];
        r->esc_out[i] = eo;
    }
    free(Q);
    free(W);
    free(Wg);
    free(Xs);
    free(Arr);
    free(L);
    free(first);
    return 0;
}

/* The preselected maximum number of couplings (Sec. 3: TURSCA keeps a
 * fixed count of the largest couplings instead of a threshold).  Every chain
 * (j, u) with a receiver other than its source carries one coupling C; with
 * K = max_couplings the scattering graph keeps the chains whose C exceeds the
 * (K + 1)-th largest of them, so exactly K are kept when that value is not
 * tied with the K-th (a tie at the boundary drops the whole tied group).
 * K at or above the count keeps every chain.  Returns the threshold for the
 * C > c_min rule: 0 for no selection, the smallest positive double when the
 * (K + 1)-th largest coupling is 0 (the zero couplings go). */
static int orc_cmp_desc(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? 1 : (x > y ? -1 : 0);
}

static double orc_topk_threshold(const orc_desc *d, const orc_result *r, const double *mu_e,
                                 const double *mus, long *n_couplings) {
    int na = r->n_atm, nn = r->n_nodes, nd = r->n_dirs, ngd = r->n_gdirs;
    double *all = malloc(sizeof(double) * ((size_t)na * nd + (size_t)r->n_ground * ngd));
    long n = 0;
    orc_chain *ch = malloc(sizeof(orc_chain));
    for (int j = 0; j < nn; ++j) {
        int ndir = j < na ? nd : ngd;
        double mus_src = j < na ? mus[j] : r->mu_s_lamb;
        for (int u = 0; u < ndir; ++u) {
            if (j < na)
                orc_atm_chain(d, r, mu_e, j, u, ch);
            else
                orc_gnd_chain(d, r, mu_e, j - na, u, ch);
            double C = orc_coupling(r, mus, ch, mus_src);
            if (C >= 0.0) all[n++] = C;
        }
    }
    free(ch);
    *n_couplings = n;
    double thr = 0.0;
    if (d->max_couplings < n) {
        qsort(all, (size_t)n, sizeof(double), orc_cmp_desc);
        thr = all[d->max_couplings];
        if (!(thr > 0.0)) thr = 4.9406564584124654e-324; /* keep C > 0 */
    }
    free(all);
    return thr;
}

int orc_run(const orc_desc *d_in, const double *mu_a, const double *mu_s, const double *g, orc_result **out) {
#ifdef _OPENMP
    if (d_in->threads > 0) omp_set_num_threads(d_in->threads);
#endif
    if (d_in->nx < 1 || d_in->ny < 1 || d_in->nz < 1 || d_in->R < 1 || d_in->R > 2 || d_in->M < 8 || d_in->S < 1)
        return 1;
    if ((d_in->flags & ORC_ANISO) && (d_in->c_min > 0.0 || d_in->max_couplings > 0))
        return 2; /* not combined with coupling selection */
    if (d_in->max_couplings < 0 || (d_in->max_couplings > 0 && d_in->c_min > 0.0)) return 3;
    orc_desc dsel = *d_in; /* c_min replaced by the threshold of a preselected count */
    const orc_desc *d = &dsel;
    orc_result *r = calloc(1, sizeof(orc_result));
    int nx = d->nx, ny = d->ny, nz = d->nz, S = d->S;
    int na = nx * ny * nz, ng = nx * ny, nn = na + ng;
    r->n_atm = na;
    r->n_ground = ng;
    r->n_nodes = nn;
    orc_make_dirs(d, r);
    int nd = r->n_dirs, ngd = r->n_gdirs;
    r->q_sun = calloc((size_t)S * nd, sizeof(double));
    orc_quadrature(d, g, r);

    /* fields */
    double *mus = calloc(na, sizeof(double)), *mue = calloc(na, sizeof(double)), *om = calloc(na, sizeof(double));
    double mus_max = 0.0;
    for (int i = 0; i < na; ++i) {
        double s = 0.0;
        for (int sp = 0; sp < S; ++sp) s += mu_s[(size_t)sp * na + i];
        mus[i] = s;
        mue[i] = mu_a[i] + s;
        om[i] = mue[i] > 0.0 ? s / mue[i] : 0.0;
        if (s > mus_max) mus_max = s;
    }
    /* Lambertian surface nodes couple with mu_s^Lamb = A max mu_s (Sec. 3) */
    r->mu_s_lamb = d->albedo * mus_max;
    if (d_in->max_couplings > 0) dsel.c_min = orc_topk_threshold(d_in, r, mue, mus, &r->n_couplings);
    r->c_min_used = dsel.c_min;

    double mu0 = cos(d->sza * ORC_PI / 180.0);
    double f0 = d->f0;
    double area = d->hx * d->hy;

    /* direct source: sun transmittance at each voxel's top-face centre and at
     * each ground point; first-order scattered power (S_a of Sec. 2, lumped
     * over the voxel with the layer-exact top-face reading) */
    r->tsun = calloc(nn, sizeof(double));
    r->e1 = calloc(nn, sizeof(double));
#pragma omp parallel for schedule(dynamic, 64)
    for (int i = 0; i < nn; ++i) {
        double P[3];
        if (i < na) {
            int iz = i / (nx * ny), iy = (i / nx) % ny, ix = i % nx;
            P[0] = ix + 0.5;
            P[1] = iy + 0.5;
            P[2] = iz + 1.0;
        } else {
            int c = i - na;
            P[0] = c % nx + 0.5;
            P[1] = c / nx + 0.5;
            P[2] = 0.0;
        }
        double T;
        orc_ray_sun(d, mue, P, &T);
        r->tsun[i] = T;
        if (i < na)
            r->e1[i] = om[i] * f0 * mu0 * area * T * (-expm1(-mue[i] * d->hz / mu0));
        else
            r->e1[i] = d->albedo * f0 * mu0 * area * T;
    }

    /* chains and per-source weights */
    int cap_a = 0, cap_g = 0;
    for (int u = 0; u < nd; ++u) cap_a += r->kmax[u] + 5;
    for (int k = 0; k < ngd; ++k) cap_g += r->gdir_nmem[k] + 1;
    size_t cap = (size_t)na * cap_a + (size_t)ng * cap_g;
    int *t_row = malloc(sizeof(int) * cap), *t_col = malloc(sizeof(int) * cap);
    int16_t *t_dir = malloc(sizeof(int16_t) * cap);
    int8_t *t_k = malloc(sizeof(int8_t) * cap);
    double *t_dep = malloc(sizeof(double) * cap), *t_dsun = malloc(sizeof(double) * cap);
    const int aniso = (d->flags & ORC_ANISO) != 0;
    double *t_P = aniso ? malloc(sizeof(double) * cap) : NULL;
    if (aniso) {
        r->chain_C = calloc((size_t)nn * nd, sizeof(double));
        r->chain_E = calloc((size_t)nn * nd, sizeof(double));
    }
    int *t_cnt = calloc(nn, sizeof(int));
    r->z_iso = calloc(nn, sizeof(double));
    r->z_sun = calloc(nn, sizeof(double));
    r->esc_iso = calloc(nn, sizeof(double));
    r->esc_sun = calloc(nn, sizeof(double));

    long n_cpl_all = 0, n_kpt_all = 0;
#pragma omp parallel
    {
        long n_cpl = 0, n_kpt = 0;
        orc_chain *ch = malloc(sizeof(orc_chain) * ORC_MAXDIR);
        double qs[ORC_MAXDIR], ci[ORC_MAXDIR], cs[ORC_MAXDIR];
        /* per-source quadrature after coupling selection */
        double qsel[ORC_MAXDIR];
        double *qsun_sel = malloc(sizeof(double) * (size_t)S * ORC_MAXDIR);
        int kept[ORC_MAXDIR];
#pragma omp for schedule(dynamic, 32)
        for (int j = 0; j < nn; ++j) {
            size_t base;
            int ndir;
            const double *qi;
            if (j < na) {
                base = (size_t)j * cap_a;
                ndir = nd;
                for (int u = 0; u < nd; ++u) orc_atm_chain(d, r, mue, j, u, &ch[u]);
                const double *qsun_j = r->q_sun;
                qi = r->q_iso;
                if (orc_select(d, r, mus, ch, nd, mus[j], kept) > 0) {
                    orc_partition_kept(d, r, g, 0, kept, qsel, qsun_sel);
                    qi = qsel;
                    qsun_j = qsun_sel;
                }
                /* q^sun_{j,u}: species mixture of the source's phase function */
                for (int u = 0; u < nd; ++u) {
                    double acc = 0.0;
                    for (int sp = 0; sp < S; ++sp) {
                        double w = mus[j] > 0.0 ? mu_s[(size_t)sp * na + j] / mus[j] : 1.0 / S;
                        acc += w * qsun_j[sp * nd + u];
                    }
                    qs[u] = acc;
                }
                orc_source_weights(d, r, mus, qi, nd, ch, 0, mus[j], ci, &r->z_iso[j]);
                orc_source_weights(d, r, mus, qs, nd, ch, 0, mus[j], cs, &r->z_sun[j]);
            } else {
                base = (size_t)na * cap_a + (size_t)(j - na) * cap_g;
                ndir = ngd;
                for (int k = 0; k < ngd; ++k) orc_gnd_chain(d, r, mue, j - na, k, &ch[k]);
                qi = r->q_lamb;
                if (orc_select(d, r, mus, ch, ngd, r->mu_s_lamb, kept) > 0) {
                    orc_partition_kept(d, r, g, 1, kept, qsel, NULL);
                    qi = qsel;
                }
                /* Lambertian re-emission forgets the incoming direction: the
                 * sun-lit and the diffusely lit ground share one quadrature */
                for (int k = 0; k < ngd; ++k) qs[k] = qi[k];
                orc_source_weights(d, r, mus, qi, ngd, ch, 1, r->mu_s_lamb, ci, &r->z_iso[j]);
                for (int k = 0; k < ngd; ++k) cs[k] = ci[k];
                r->z_sun[j] = r->z_iso[j];
            }
            if (aniso)
                for (int u = 0; u < ndir; ++u) {
                    r->chain_C[(size_t)j * nd + u] = orc_coupling(r, mus, &ch[u], j < na ? mus[j] : r->mu_s_lamb);
                    r->chain_E[(size_t)j * nd + u] = ch[u].escape;
                }
            for (int u = 0; u < ndir; ++u)
                if (orc_coupling(r, mus, &ch[u], j < na ? mus[j] : r->mu_s_lamb) >= 0.0) {
                    n_cpl++;
                    n_kpt += kept[u];
                }
            int cnt = 0;
            double ei = 0.0, es = 0.0;
            for (int u = 0; u < ndir; ++u) {
                double wi = qi[u] * ci[u], ws = qs[u] * cs[u];
                ei += wi * ch[u].escape;
                es += ws * ch[u].escape;
                for (int t = 0; t < ch[u].ndep; ++t) {
                    size_t e = base + cnt++;
                    t_row[e] = ch[u].dep[t].node;
                    t_col[e] = j;
                    t_dir[e] = (int16_t)(j < na ? u : nd + u);
                    t_k[e] = (int8_t)ch[u].dep[t].k;
                    t_dep[e] = wi * ch[u].dep[t].P;
                    t_dsun[e] = ws * ch[u].dep[t].P;
                    if (aniso) t_P[e] = ch[u].dep[t].P;
                }
            }
            r->esc_iso[j] = ei;
            r->esc_sun[j] = es;
            t_cnt[j] = cnt;
        }
        free(ch);
        free(qsun_sel);
#pragma omp atomic
        n_cpl_all += n_cpl;
#pragma omp atomic
        n_kpt_all += n_kpt;
    }
    r->n_couplings = n_cpl_all;
    r->n_kept = n_kpt_all;

    /* gather into row-major order (stable: by source, then direction) */
    int *rowcnt = calloc(nn + 1, sizeof(int));
    long tot = 0;
    for (int j = 0; j < nn; ++j) {
        size_t base = j < na ? (size_t)j * cap_a : (size_t)na * cap_a + (size_t)(j - na) * cap_g;
        for (int t = 0; t < t_cnt[j]; ++t) rowcnt[t_row[base + t] + 1]++;
        tot += t_cnt[j];
    }
    for (int i = 0; i < nn; ++i) rowcnt[i + 1] += rowcnt[i];
    r->n_slots = tot;
    r->slot_row = malloc(sizeof(int) * tot);
    r->slot_col = malloc(sizeof(int) * tot);
    r->slot_dir = malloc(sizeof(int16_t) * tot);
    r->slot_k = malloc(sizeof(int8_t) * tot);
    r->slot_dep = malloc(sizeof(double) * tot);
    r->slot_depsun = malloc(sizeof(double) * tot);
    if (aniso) r->slot_P = malloc(sizeof(double) * tot);
    r->slot_val = malloc(sizeof(double) * tot);
    r->slot_valsun = malloc(sizeof(double) * tot);
    int *fill = malloc(sizeof(int) * nn);
    memcpy(fill, rowcnt, sizeof(int) * nn);
    for (int j = 0; j < nn; ++j) {
        size_t base = j < na ? (size_t)j * cap_a : (size_t)na * cap_a + (size_t)(j - na) * cap_g;
        for (int t = 0; t < t_cnt[j]; ++t) {
            size_t src = base + t;
            int row = t_row[src];
            long e = fill[row]++;
            double rho = row < na ? om[row] : d->albedo;
            r->slot_row[e] = row;
            r->slot_col[e] = t_col[src];
            r->slot_dir[e] = t_dir[src];
            r->slot_k[e] = t_k[src];
            r->slot_dep[e] = t_dep[src];
            r->slot_depsun[e] = t_dsun[src];
            if (aniso) r->slot_P[e] = t_P[src];
            r->slot_val[e] = rho * t_dep[src];
            r->slot_valsun[e] = rho * t_dsun[src];
        }
    }
    free(fill);
    free(t_row);
    free(t_col);
    free(t_dir);
    free(t_k);
    free(t_dep);
    free(t_dsun);
    free(t_P);
    free(t_cnt);

    /* s = K^sun e1 */
    r->s = calloc(nn, sizeof(double));
    r->x = calloc(nn, sizeof(double));
    int single = (d->flags & ORC_SINGLE_SCATTER) != 0;
    if (!single) {
#pragma omp parallel for schedule(static)
        for (int i = 0; i < nn; ++i) {
            double acc = 0.0;
            for (int e = rowcnt[i]; e < rowcnt[i + 1]; ++e) acc += r->slot_valsun[e] * r->e1[r->slot_col[e]];
            r->s[i] = acc;
        }
    }
    if (d->flags & ORC_NO_SOLVE) {
        free(rowcnt);
        free(mus);
        free(mue);
        free(om);
        *out = r;
        return 0;
    }
    if (!single) {
        if (aniso) {
            if (orc_aniso(d, r, g, mu_s, mus, om, rowcnt) != 0) {
                free(rowcnt);
                free(mus);
                free(mue);
                free(om);
                orc_free(r);
                return 3;
            }
        } else {
            orc_gmres(d, r, rowcnt, r->slot_col, r->slot_val);
        }
    }

    /* emission toward the instrument */
    double s0[3], vv[3];
    orc_sun_dir(d, s0);
    orc_view_dir(d, vv);
    double mus0v = s0[0] * vv[0] + s0[1] * vv[1] + s0[2] * vv[2];
    double ucos[ORC_MAXDIR + ORC_MAXGDIR];
    for (int u = 0; u < nd; ++u) {
        double uh[3], L;
        orc_atm_dir(d, r, u, uh, &L);
        ucos[u] = uh[0] * vv[0] + uh[1] * vv[1] + uh[2] * vv[2];
    }
    for (int k = 0; k < ngd; ++k) {
        double uh[3];
        orc_gnd_dir(d, r, k, uh);
        ucos[nd + k] = uh[0] * vv[0] + uh[1] * vv[1] + uh[2] * vv[2];
    }
    r->emis1 = calloc(na, sizeof(double));
    r->emis_sun = calloc(na, sizeof(double));
    r->emis_ms = calloc(na, sizeof(double));
    double *emis = calloc(na, sizeof(double));
#pragma omp parallel for schedule(static)
    for (int i = 0; i < na; ++i) {
        /* Theta_i: mixture of the species' HG functions weighted by mu_s */
        double w[16];
        for (int sp = 0; sp < S; ++sp) w[sp] = mus[i] > 0.0 ? mu_s[(size_t)sp * na + i] / mus[i] : 1.0 / S;
        double th0 = 0.0;
        for (int sp = 0; sp < S; ++sp) th0 += w[sp] * orc_hg(g[sp], mus0v);
        r->emis1[i] = r->e1[i] * th0;
        double es = 0.0, em = 0.0;
        if (!single)
            for (int e = rowcnt[i]; e < rowcnt[i + 1]; ++e) {
                double th = 0.0;
                for (int sp = 0; sp < S; ++sp) th += w[sp] * orc_hg(g[sp], ucos[r->slot_dir[e]]);
                es += th * r->slot_valsun[e] * r->e1[r->slot_col[e]];
                if (!aniso) em += th * r->slot_val[e] * r->x[r->slot_col[e]];
            }
        if (!single && aniso) {
            /* every arrival direction's scattered power, less the first-order part */
            double et = 0.0;
            for (int wv = 0; wv < nd + ngd; ++wv) {
                double th = 0.0;
                for (int sp = 0; sp < S; ++sp) th += w[sp] * orc_hg(g[sp], ucos[wv]);
                et += th * r->X[(size_t)i * (nd + ngd) + wv];
            }
            em = et - es;
        }
        r->emis_sun[i] = es;
        r->emis_ms[i] = em;
        emis[i] = r->emis1[i] + es + em;
    }

    /* pixels */
    int npx = d->npx, npy = d->npy;
    r->rad = calloc((size_t)npx * npy, sizeof(double));
    r->refl = calloc((size_t)npx * npy, sizeof(double));
    double vol = d->hx * d->hy * d->hz;
    double H = nz * d->hz;
#pragma omp parallel for schedule(dynamic, 16)
    for (int p = 0; p < npx * npy; ++p) {
        int a = p % npx, b = p / npx;
        double gx = (a + 0.5) * nx / (double)npx, gy = (b + 0.5) * ny / (double)npy; /* cell units */
        double len = H / vv[2];
        double P[3] = {gx + len * vv[0] / d->hx, gy + len * vv[1] / d->hy, (double)nz};
        double V[3] = {-vv[0] / d->hx, -vv[1] / d->hy, -vv[2] / d->hz};
        orc_los ctx = {mue, emis, vol, 1.0, 0.0, 0.0};
        orc_dda(d, mue, P, V, len, 1.0, los_seg, &ctx);
        int cx = imod((int)floor(gx), nx), cy = imod((int)floor(gy), ny);
        int c = na + cy * nx + cx;
        double Lg = exp(-ctx.tau) * (r->e1[c] + r->x[c]) / (ORC_PI * area);
        r->rad[p] = ctx.L + Lg;
        r->refl[p] = ORC_PI * r->rad[p] / (mu0 * f0);
    }
    free(emis);
    free(rowcnt);
    free(mus);
    free(mue);
    free(om);
    *out = r;
    return 0;
}

void orc_free(orc_result *r) {
    if (!r) return;
    free(r->slot_P);
    free(r->chain_C);
    free(r->chain_E);
    free(r->X);
    free(r->arrive);
    free(r->esc_out);
    free(r->q_sun);
    free(r->tsun);
    free(r->e1);
    free(r->z_iso);
    free(r->z_sun);
    free(r->esc_iso);
    free(r->esc_sun);
    free(r->slot_row);
    free(r->slot_col);
    free(r->slot_dir);
    free(r->slot_k);
    free(r->slot_dep);
    free(r->slot_depsun);
    free(r->slot_val);
    free(r->slot_valsun);
    free(r->s);
    free(r->x);
    free(r->emis1);
    free(r->emis_sun);
    free(r->emis_ms);
    free(r->rad);
    free(r->refl);
    free(r);
}

/* Optical depth of one straight segment through mu_e (cell-unit start P,    */
/* cell-unit direction V per unit t, t in [0, tend], physical length per t). */
double orc_tau_segment(const orc_desc *d, const double *mu_e, const double *P, const double *V, double tend,
                       double lphys) {
    return orc_dda(d, mu_e, P, V, tend, lphys, NULL, NULL);
}

/* Quadrature weights of one source over a kept set of directions (coupling
 * selection): ground = 0 for the atmospheric set (qi[n_dirs], qsun[S][n_dirs]),
 * 1 for the ground set (qi[n_gdirs]).  Returns the number of directions. */
int orc_partition(const orc_desc *d, const double *g, int ground, const int *kept, double *qi, double *qsun) {
    orc_result *r = calloc(1, sizeof(orc_result));
    orc_make_dirs(d, r);
    int n = ground ? r->n_gdirs : r->n_dirs;
    orc_partition_kept(d, r, g, ground, kept, qi, qsun);
    free(r);
    return n;
}

/* Q[S][n_dirs + n_gdirs][n_dirs]: the phase quadrature by arrival direction
 * (see orc_phase_quadrature_fill); *n_dirs gets n_dirs.  Returns
 * n_dirs + n_gdirs. */
int orc_phase_quadrature(const orc_desc *d, const double *g, double *Q, int *n_dirs) {
    orc_result *r = calloc(1, sizeof(orc_result));
    orc_make_dirs(d, r);
    int nin = r->n_dirs + r->n_gdirs;
    *n_dirs = r->n_dirs;
    orc_phase_quadrature_fill(d, r, g, Q);
    free(r);
    return nin;
}

/* Fibonacci lattice point m of M (unit vector). */
void orc_fibonacci(int m, int M, double *s) { orc_fib_point(m, M, s); }

int orc_result_size(void) { return (int)sizeof(orc_result); }
int orc_desc_size(void) { return (int)sizeof(orc_desc); }

/* The edge form's fixed-point map at chosen receiver rows (for checks of a
 * solution X at sizes where the whole series does not fit): with X given for
 * every node ([n_nodes][n_dirs + n_gdirs], the arrival directions as in
 * orc_aniso), out[t][w] = F(X)(rows[t], w), where
 *   F(X)(i, w) = rho_i sum_{slots e of row i arriving along w}
 *                  (P_e L(src_e, dir_e) + depsun_e e1(src_e))
 *   L(j, u)    = sum_w' X(j, w') Q_j(w' -> u) c_j(u | w')     atmospheric j
 *   L(c, k)    = (sum_w' X(c, w')) q_lamb_k c_k                ground c
 * the same definitions orc_aniso iterates (Eq. flux_system, Eq. F_term_phase),
 * each source's leaving power built only when a chosen row needs it.
 * Returns 0, or the code of orc_run. */
int orc_aniso_rows(const orc_desc *d_in, const double *mu_a, const double *mu_s, const double *g, const double *X,
                   const int *rows, int nrows, double *out) {
    orc_desc dd = *d_in;
    dd.flags |= ORC_ANISO | ORC_NO_SOLVE;
    orc_result *r = NULL;
    int rc = orc_run(&dd, mu_a, mu_s, g, &r);
    if (rc != 0) return rc;
    const int na = r->n_atm, nn = r->n_nodes, nd = r->n_dirs, ngd = r->n_gdirs, S = dd.S, nin = nd + ngd;
    /* row ranges of the slots (sorted by row) */
    long *start = calloc((size_t)nn + 1, sizeof(long));
    for (long e = 0; e < r->n_slots; ++e) start[r->slot_row[e] + 1]++;
    for (int i = 0; i < nn; ++i) start[i + 1] += start[i];
    double *Q = malloc(sizeof(double) * (size_t)S * nin * nd);
    orc_phase_quadrature_fill(&dd, r, g, Q);
    double *mus = calloc((size_t)na, sizeof(double));
    for (int j = 0; j < na; ++j)
        for (int sp = 0; sp < S; ++sp) mus[j] += mu_s[(size_t)sp * na + j];
#pragma omp parallel for schedule(dynamic, 1)
    for (int t = 0; t < nrows; ++t) {
        const int i = rows[t];
        double *o = out + (size_t)t * nin;
        for (int w = 0; w < nin; ++w) o[w] = 0.0;
        if (i < 0 || i >= nn) continue;
        const double mue_i = i < na ? mu_a[i] + mus[i] : 0.0;
        const double rho = i < na ? (mue_i > 0.0 ? mus[i] / mue_i : 0.0) : dd.albedo;
        for (long e = start[i]; e < start[i + 1]; ++e) {
            const int j = r->slot_col[e], din = r->slot_dir[e];
            const int u = din < nd ? din : din - nd;
            /* L(j, u) from the definitions (one source, one direction) */
            double L = 0.0;
            if (j < na) {
                double q[ORC_MAXDIR], cw[ORC_MAXDIR], z, wsp[16];
                for (int sp = 0; sp < S; ++sp) wsp[sp] = mus[j] > 0.0 ? mu_s[(size_t)sp * na + j] / mus[j] : 1.0 / S;
                for (int w = 0; w < nin; ++w) {
                    const double xw = X[(size_t)j * nin + w];
                    if (xw == 0.0) continue;
                    for (int v = 0; v < nd; ++v) {
                        double acc = 0.0;
                        for (int sp = 0; sp < S; ++sp) acc += wsp[sp] * Q[((size_t)sp * nin + w) * nd + v];
                        q[v] = acc;
                    }
                    orc_route(&dd, &r->chain_C[(size_t)j * nd], q, nd, cw, &z);
                    L += xw * q[u] * cw[u];
                }
            } else {
                double cw[ORC_MAXGDIR], z, xt = 0.0;
                orc_route(&dd, &r->chain_C[(size_t)j * nd], r->q_lamb, ngd, cw, &z);
                for (int w = 0; w < nin; ++w) xt += X[(size_t)j * nin + w];
                L = xt * r->q_lamb[u] * cw[u];
            }
            o[din] += rho * (r->slot_P[e] * L + r->slot_depsun[e] * r->e1[j]);
        }
    }
    free(mus);
    free(Q);
    free(start);
    orc_free(r);
    return 0;
}
