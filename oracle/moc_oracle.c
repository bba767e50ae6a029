/*
 * moc_oracle.c -- plain FP64 CPU oracle for the 3D MOC transport sweep of
 * "Neutron particle transport 3D method of characteristic Multi GPU platform
 * Parallel Computing" (arXiv 2503.17743).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the GPU library; the only common input is the
 * seeded problem description (lattice, cross sections, track layout).
 *
 * What it computes, step by step, in the order the paper gives them:
 *   1. Flat source regions: radial regions of an axially extruded pin lattice
 *      (Sec. 2.2, extruded geometry) times uniform axial layers.  A pin cell
 *      may be refined into rings (equal areas inside the fuel circle, equal
 *      area steps out to the inscribed circle) and equal angular sectors.
 *   2. 2D cyclic tracks and their 2D segments (kept on the CPU, Sec. 3.1).
 *   3. z-stacks of 3D tracks z_i(s) = z_0 + i dz + s cot(theta) (Eq. 5); the
 *      tracks crossing each (2D segment, layer) FSR from Eqs. 6-7, the full
 *      2D-length crossings from Eqs. 9-10 with length Eq. 8, the full axial
 *      crossings with length Eq. 11, partial crossings otherwise.
 *   4. Alg. 1 loop order: for each 2D track, for each polar angle, for each
 *      track of the z-stack: generate it, trace its segments, sweep it.
 *   5. Eq. 3 attenuation per segment and group, both directions.
 *   6. Scalar flux from the track-weighted segment tallies (Eq. 4, read as
 *      the standard flat-source tally: phi = (4 pi Q + tally / V) / Sigma_t).
 *   7. Isotropic source update and power iteration on k-eff.
 *
 * Readings of points the paper leaves open (laydown, linking, tie rules) are
 * stated where they are used; they are the same conventions the GPU library
 * implements independently.  Floating point is IEEE FP64 throughout; build
 * with -ffp-contract=off so that no multiply-add is fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define TIE_EPS 1e-10      /* lattice coordinates this close to an integer are that integer */
#define SEG2D_MIN 1e-10    /* 2D intervals shorter than this (cm) are merged away */

typedef struct {
    int ncx, ncy, n_layers;
    double pitch, radius, height;
    const int *has_pin;   /* [ncy*ncx] */
    const int *mat_in;    /* [ncy*ncx*n_layers] */
    const int *mat_out;   /* [ncy*ncx*n_layers] */
    int bc[6];            /* xmin xmax ymin ymax zmin zmax: 1 reflective, 0 vacuum */
    int M, G;
    const double *sigma_t;    /* [M*G] */
    const double *sigma_s;    /* [M*G*G] from g into h */
    const double *nu_sigma_f; /* [M*G] */
    const double *chi;        /* [M*G] */
    const double *ext_source; /* [M*G] or NULL */
    int n_azim, n_polar;
    double radial_spacing, axial_spacing;
    int n_threads;
    int light;  /* 1: tracks and segments only (no links, boundary fluxes or
                   volumes): for sampled checks of problems too large to solve */
    int fuel_rings, mod_rings, sectors;  /* pin-cell refinement (0 read as 1, 0, 1) */
    const double *layer_z;  /* [n_layers + 1] layer planes from 0 to height, or NULL
                               (equal layers); each a whole number of axial spacings */
} orc_input;

/* faces */
enum { F_XMIN = 0, F_XMAX = 1, F_YMIN = 2, F_YMAX = 3, F_ZMIN = 4, F_ZMAX = 5 };

typedef struct {
    /* inputs */
    int ncx, ncy, nl, M, G, A, P, nthreads;
    double pitch, radius, H;
    int *has_pin, *mat_in, *mat_out;
    int bc[6];
    double *st, *ss, *nsf, *chi, *src;
    /* FSRs */
    double Wx, Wy;
    int nreg, nfsr;
    int nfuel_rings, ncirc, nsec;  /* pin cells: circles (fuel ones first), sectors */
    double circ_r2[130];           /* squared radii of the circles, increasing */
    int *reg_base;      /* per cell */
    int *fsr_mat;       /* per FSR */
    int Nz, cpl;      /* cpl: lattice cells per layer (0 when the layers differ) */
    long *lplane;     /* [nl + 1] integer part of each layer plane in lattice units, z / dz */
    double *kplane;   /* [nl + 1] each layer plane in lattice units (any mesh) */
    double *qplane;   /* [nl + 1] its fractional part, the pfrac entry itself when nonzero */
    double *pfrac;    /* distinct fractional parts of the planes, ascending */
    int npfrac;
    double dz;
    /* azimuth pairs m = 0..nq-1 */
    int nq;
    long *nx, *ny, *gg, *Mcyc;
    double *phi_eff, *span, *deff, *lu;
    /* polar: Ph per hemisphere; per (m, ph) */
    int Ph;
    double *mu_gl, *w_gl;
    long *cpol;
    double *cot, *sinp, *cosp;
    /* 2D tracks */
    int nt;
    int *a_off;                 /* first track of azimuth a, size A/2+1 */
    int *t_azim, *t_sface, *t_sk, *t_eface, *t_ek;
    long *t_steps, *t_M;
    double *t_x0, *t_y0, *t_len;
    int *succ_t[2], *succ_s[2]; /* successor (track, sense) after leaving in sense 0 (fwd) / 1 (bwd) */
    int kmax;
    int *start_tab, *end_tab;   /* [(a*4+face)*kmax + k] -> track */
    /* 2D segments: CSR, boundary positions spos[soff[t]+t ... +nb] */
    long *soff;
    int *sreg;
    double *slen, *spos;
    /* stacks (t, p): p in [0, P); p < Ph up (cot > 0), p >= Ph mirrored down */
    long *stk_imin, *stk_n, *stk_slot;
    long n3d;
    long *dest;                 /* [n3d*2] destination (slot*2+sense) or -1 (leak) */
    double *W;                  /* per (m, ph): track weight w_d * dA_d */
    /* state */
    double *V, *phi, *psi0, *psi1, k;
    double last_leak, last_res;
    double *fiss_old;
} orc_t;

static char g_err[256];
static void set_err(char *err, int len, const char *msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
    if (err && len > 0) snprintf(err, (size_t)len, "%s", msg);
}
const char *orc_last_error(void) { return g_err; }

static long gcd_l(long a, long b) { while (b) { long t = a % b; a = b; b = t; } return a; }
static long mod_l(long a, long m) { long r = a % m; return r < 0 ? r + m : r; }

/* Gauss-Legendre nodes/weights on (-1, 1) by Newton iteration on P_n. */
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; i++) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; j++) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1.0);
            double dz = p1 / pp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

static double snap(double z) {
    double r = nearbyint(z);
    return fabs(z - r) <= TIE_EPS ? r : z;
}

/* Layer planes off the axial lattice (a local axial mesh, Sec. 2.2).  A
 * lattice coordinate u is kept as its integer part n and fractional part f,
 * and a fraction within TIE_EPS of a plane's fractional part is replaced by
 * that plane's fraction (the same double), so that "u lies on the plane" and
 * "u lies below it" are exact comparisons of integers and of equal doubles,
 * decided the same way by any implementation of the same arithmetic and for
 * integer parts of any size. */
static void split_coord(const double *pfrac, int npfrac, double z, long *n, double *f) {
    z = snap(z);
    double fl = floor(z), fr = z - fl;
    for (int q = 0; q < npfrac; q++)
        if (fabs(fr - pfrac[q]) <= TIE_EPS) { fr = pfrac[q]; break; }
    *n = (long)fl;
    *f = fr;
}

/* u < v for split coordinates */
static int coord_lt(long un, double uf, long vn, double vf) {
    return un < vn || (un == vn && uf < vf);
}

/* ------------------------------------------------------------------------
 * 2D cyclic tracking (kept on the CPU by the paper, Sec. 3.1).
 *
 * Reading of the unspecified laydown (textbook cyclic tracking): for the
 * desired angle phi_m = 2 pi (m + 1/2) / A in the first quadrant,
 * nx = ceil(Wx sin(phi)/delta), ny = ceil(Wy cos(phi)/delta),
 * tan(phi_eff) = (Wy nx)/(Wx ny), delta_eff = (Wx/nx) sin(phi_eff).  Tracks
 * start at the half-offset points of the bottom face (x = (k+1/2) Wx/nx) and of
 * the side face (y = (k+1/2) Wy/ny).  In the scaled coordinates
 * X = x / (Wx/2nx), Y = y / (Wy/2ny) every track is a 45 degree diagonal
 * between integer points, which makes every end point, link and cycle
 * position an exact integer.
 * ---------------------------------------------------------------------- */

static void track_end(long nxm, long nym, int right, int sface, long k,
                      long *X1, long *Y1, long *t) {
    long X0, Y0;
    if (sface == F_YMIN) { X0 = 2 * k + 1; Y0 = 0; }
    else if (sface == F_XMIN) { X0 = 0; Y0 = 2 * k + 1; }
    else { X0 = 2 * nxm; Y0 = 2 * k + 1; }
    long lim_x = right ? (2 * nxm - X0) : X0;
    long lim_y = 2 * nym - Y0;
    long tt = lim_x < lim_y ? lim_x : lim_y;
    *t = tt;
    *X1 = right ? X0 + tt : X0 - tt;
    *Y1 = Y0 + tt;
}

/* index of the track of azimuth a that starts (want_start) or ends at (face, k),
 * from tables filled by scanning every track's end points */
static int find_track(orc_t *o, int a, int face, int k, int want_start) {
    if (k < 0 || k >= o->kmax) return -1;
    const int *tab = want_start ? o->start_tab : o->end_tab;
    return tab[((size_t)a * 4 + face) * o->kmax + k];
}

static int build_2d(orc_t *o, char *err, int errlen) {
    int A = o->A, nq = o->nq;
    o->a_off = calloc((size_t)A / 2 + 1, sizeof(int));
    int total = 0;
    for (int a = 0; a < A / 2; a++) {
        int m = a < nq ? a : A / 2 - 1 - a;
        o->a_off[a] = total;
        total += (int)(o->nx[m] + o->ny[m]);
    }
    o->a_off[A / 2] = total;
    o->nt = total;
    int nt = total;
    o->t_azim = calloc(nt, sizeof(int));
    o->t_sface = calloc(nt, sizeof(int));
    o->t_sk = calloc(nt, sizeof(int));
    o->t_eface = calloc(nt, sizeof(int));
    o->t_ek = calloc(nt, sizeof(int));
    o->t_steps = calloc(nt, sizeof(long));
    o->t_M = calloc(nt, sizeof(long));
    o->t_x0 = calloc(nt, sizeof(double));
    o->t_y0 = calloc(nt, sizeof(double));
    o->t_len = calloc(nt, sizeof(double));
    for (int s = 0; s < 2; s++) {
        o->succ_t[s] = calloc(nt, sizeof(int));
        o->succ_s[s] = calloc(nt, sizeof(int));
    }
    for (int a = 0; a < A / 2; a++) {
        int m = a < nq ? a : A / 2 - 1 - a;
        int right = a < nq;
        long nxm = o->nx[m], nym = o->ny[m];
        int t = o->a_off[a];
        for (long k = 0; k < nxm + nym; k++, t++) {
            int sface = k < nxm ? F_YMIN : (right ? F_XMIN : F_XMAX);
            long kk = k < nxm ? k : k - nxm;
            long X1, Y1, tt;
            track_end(nxm, nym, right, sface, kk, &X1, &Y1, &tt);
            o->t_azim[t] = a;
            o->t_sface[t] = sface;
            o->t_sk[t] = (int)kk;
            if (Y1 == 2 * nym) { o->t_eface[t] = F_YMAX; o->t_ek[t] = (int)((X1 - 1) / 2); }
            else if (X1 == 2 * nxm) { o->t_eface[t] = F_XMAX; o->t_ek[t] = (int)((Y1 - 1) / 2); }
            else { o->t_eface[t] = F_XMIN; o->t_ek[t] = (int)((Y1 - 1) / 2); }
            o->t_steps[t] = tt;
            double ux = o->Wx / (2.0 * nxm), uy = o->Wy / (2.0 * nym);
            if (sface == F_YMIN) { o->t_x0[t] = (2 * kk + 1) * ux; o->t_y0[t] = 0.0; }
            else if (sface == F_XMIN) { o->t_x0[t] = 0.0; o->t_y0[t] = (2 * kk + 1) * uy; }
            else { o->t_x0[t] = o->Wx; o->t_y0[t] = (2 * kk + 1) * uy; }
            o->t_len[t] = (double)tt * o->lu[m];
        }
    }
    o->kmax = 1;
    for (int m = 0; m < nq; m++) {
        if (o->nx[m] > o->kmax) o->kmax = (int)o->nx[m];
        if (o->ny[m] > o->kmax) o->kmax = (int)o->ny[m];
    }
    size_t ntab = (size_t)(A / 2) * 4 * o->kmax;
    o->start_tab = malloc(sizeof(int) * ntab);
    o->end_tab = malloc(sizeof(int) * ntab);
    for (size_t q = 0; q < ntab; q++) o->start_tab[q] = o->end_tab[q] = -1;
    for (int t = 0; t < nt; t++) {
        int a = o->t_azim[t];
        o->start_tab[((size_t)a * 4 + o->t_sface[t]) * o->kmax + o->t_sk[t]] = t;
        o->end_tab[((size_t)a * 4 + o->t_eface[t]) * o->kmax + o->t_ek[t]] = t;
    }
    /* reflective successors: reflect the direction at the face it leaves by */
    for (int t = 0; t < nt; t++) {
        int a = o->t_azim[t];
        int m = a < nq ? a : A / 2 - 1 - a;
        int dxs = a < nq ? 1 : -1;  /* direction of the forward sense in (X, Y) */
        for (int sense = 0; sense < 2; sense++) {
            int face = sense == 0 ? o->t_eface[t] : o->t_sface[t];
            int k = sense == 0 ? o->t_ek[t] : o->t_sk[t];
            int dx = sense == 0 ? dxs : -dxs, dy = sense == 0 ? 1 : -1;
            if (face == F_XMIN || face == F_XMAX) dx = -dx; else dy = -dy;
            int a2, want_start, s2;
            if (dy > 0) { a2 = dx > 0 ? m : A / 2 - 1 - m; want_start = 1; s2 = 0; }
            else { a2 = (-dx) > 0 ? m : A / 2 - 1 - m; want_start = 0; s2 = 1; }
            int t2 = find_track(o, a2, face, k, want_start);
            if (t2 < 0) { set_err(err, errlen, "2D link not found"); return -1; }
            o->succ_t[sense][t] = t2;
            o->succ_s[sense][t] = s2;
        }
    }
    /* cycles: positions in half-unit steps, origin at the lowest-numbered track
     * traversed forward; a track traversed backward at position p gets the
     * position of its start in the reversed cycle, Mcyc - p - steps. */
    char *vis = calloc(nt, 1);
    for (int m = 0; m < nq; m++) {
        int aa[2] = {m, A / 2 - 1 - m};   /* m < A/2-1-m: increasing track number */
        for (int side = 0; side < 2; side++) {
            for (int t0 = o->a_off[aa[side]]; t0 < o->a_off[aa[side] + 1]; t0++) {
                if (vis[t0]) continue;
                long pos = 0;
                int t = t0, s = 0;
                do {
                    if (vis[t]) { set_err(err, errlen, "track visited twice in cycle"); free(vis); return -1; }
                    vis[t] = 1;
                    o->t_M[t] = s == 0 ? pos : mod_l(o->Mcyc[m] - pos - o->t_steps[t], o->Mcyc[m]);
                    pos += o->t_steps[t];
                    int tn = o->succ_t[s][t], sn = o->succ_s[s][t];
                    t = tn; s = sn;
                } while (!(t == t0 && s == 0));
                if (pos != o->Mcyc[m]) { set_err(err, errlen, "cycle length mismatch"); free(vis); return -1; }
            }
        }
    }
    free(vis);
    return 0;
}

/* 2D segments of one track: all crossings with cell lines and pin circles,
 * sorted; tiny intervals merged away (right breakpoint removed, or the left
 * one for the last interval); each interval classified by its midpoint. */
static int region_at(orc_t *o, double x, double y) {
    int cx = (int)floor(x / o->pitch), cy = (int)floor(y / o->pitch);
    if (cx < 0) cx = 0;
    if (cx >= o->ncx) cx = o->ncx - 1;
    if (cy < 0) cy = 0;
    if (cy >= o->ncy) cy = o->ncy - 1;
    int c = cy * o->ncx + cx;
    if (!o->has_pin[c]) return o->reg_base[c];
    double ccx = (cx + 0.5) * o->pitch, ccy = (cy + 0.5) * o->pitch;
    double d2 = (x - ccx) * (x - ccx) + (y - ccy) * (y - ccy);
    int ring = o->ncirc;
    for (int k = o->ncirc - 1; k >= 0; k--)
        if (d2 < o->circ_r2[k]) ring = k;
    int sec = 0;
    if (o->nsec > 1) {
        double ang = atan2(y - ccy, x - ccx);
        if (ang < 0.0) ang += 2.0 * ORC_PI;
        sec = (int)floor(ang / (2.0 * ORC_PI / o->nsec));
        if (sec >= o->nsec) sec = o->nsec - 1;
    }
    return o->reg_base[c] + ring * o->nsec + sec;
}

static int cmp_dbl(const void *a, const void *b) {
    double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

static int trace_track(orc_t *o, int t, double **bp_out, int *nbp_out) {
    int a = o->t_azim[t];
    int m = a < o->nq ? a : o->A / 2 - 1 - a;
    double ux = o->Wx / (2.0 * o->nx[m]), uy = o->Wy / (2.0 * o->ny[m]);
    double dx = (a < o->nq ? ux : -ux) / o->lu[m], dy = uy / o->lu[m];
    double x0 = o->t_x0[t], y0 = o->t_y0[t], L = o->t_len[t];
    int cap = 2 * (o->ncx + o->ncy) + 8;
    double *bp = malloc(sizeof(double) * (size_t)(cap * (2 * o->ncirc + o->nsec + 2)));
    int n = 0;
    bp[n++] = 0.0;
    bp[n++] = L;
    for (int j = 1; j < o->ncx; j++) {
        double tt = (j * o->pitch - x0) / dx;
        if (tt > 0.0 && tt < L) bp[n++] = tt;
    }
    for (int j = 1; j < o->ncy; j++) {
        double tt = (j * o->pitch - y0) / dy;
        if (tt > 0.0 && tt < L) bp[n++] = tt;
    }
    qsort(bp, (size_t)n, sizeof(double), cmp_dbl);
    /* circles of the pin cells between consecutive line crossings */
    int nlines = n;
    for (int i = 0; i + 1 < nlines; i++) {
        double tm = 0.5 * (bp[i] + bp[i + 1]);
        double xm = x0 + tm * dx, ym = y0 + tm * dy;
        int cx = (int)floor(xm / o->pitch), cy = (int)floor(ym / o->pitch);
        if (cx < 0 || cx >= o->ncx || cy < 0 || cy >= o->ncy) continue;
        if (!o->has_pin[cy * o->ncx + cx]) continue;
        double ccx = (cx + 0.5) * o->pitch, ccy = (cy + 0.5) * o->pitch;
        double fx = x0 - ccx, fy = y0 - ccy;
        double b = fx * dx + fy * dy;
        for (int k = 0; k < o->ncirc; k++) {
            double cc = fx * fx + fy * fy - o->circ_r2[k];
            double disc = b * b - cc;
            if (disc <= 0.0) continue;
            double sq = sqrt(disc);
            double t1 = -b - sq, t2 = -b + sq;
            if (t1 > bp[i] && t1 < bp[i + 1]) bp[n++] = t1;
            if (t2 > bp[i] && t2 < bp[i + 1]) bp[n++] = t2;
        }
        /* sector boundaries: the half-lines from the centre at the angles
           2 pi s / S; the chord meets the full line of angle th where the
           cross product with (cos th, sin th) vanishes, and that point is on
           the half-line when its projection on it is not negative */
        for (int s = 0; o->nsec > 1 && s < o->nsec; s++) {
            double th = 2.0 * ORC_PI * s / o->nsec;
            double ux = cos(th), uy = sin(th);
            double cr = dx * uy - dy * ux;
            if (cr == 0.0) continue;
            double tt = (fy * ux - fx * uy) / cr;
            if (!(tt > bp[i] && tt < bp[i + 1])) continue;
            if ((fx + tt * dx) * ux + (fy + tt * dy) * uy >= 0.0) bp[n++] = tt;
        }
    }
    qsort(bp, (size_t)n, sizeof(double), cmp_dbl);
    /* merge tiny intervals */
    int changed = 1;
    while (changed && n > 2) {
        changed = 0;
        for (int i = 0; i + 1 < n; i++) {
            if (bp[i + 1] - bp[i] < SEG2D_MIN) {
                int del = (i + 1 == n - 1) ? i : i + 1;
                if (del == 0) del = 1;
                memmove(bp + del, bp + del + 1, sizeof(double) * (size_t)(n - del - 1));
                n--;
                changed = 1;
                break;
            }
        }
    }
    *bp_out = bp;
    *nbp_out = n;
    return 0;
}

static int build_2d_segments(orc_t *o) {
    int nt = o->nt;
    double **bps = malloc(sizeof(double *) * (size_t)nt);
    int *nbs = malloc(sizeof(int) * (size_t)nt);
    long total = 0;
    for (int t = 0; t < nt; t++) {
        trace_track(o, t, &bps[t], &nbs[t]);
        total += nbs[t] - 1;
    }
    o->soff = malloc(sizeof(long) * (size_t)(nt + 1));
    o->sreg = malloc(sizeof(int) * (size_t)total);
    o->slen = malloc(sizeof(double) * (size_t)total);
    o->spos = malloc(sizeof(double) * (size_t)(total + nt));
    long off = 0;
    for (int t = 0; t < nt; t++) {
        int a = o->t_azim[t];
        int m = a < o->nq ? a : o->A / 2 - 1 - a;
        double ux = o->Wx / (2.0 * o->nx[m]), uy = o->Wy / (2.0 * o->ny[m]);
        double dx = (a < o->nq ? ux : -ux) / o->lu[m], dy = uy / o->lu[m];
        o->soff[t] = off;
        int nb = nbs[t] - 1;
        for (int j = 0; j < nb; j++) {
            double tm = 0.5 * (bps[t][j] + bps[t][j + 1]);
            o->sreg[off + j] = region_at(o, o->t_x0[t] + tm * dx, o->t_y0[t] + tm * dy);
            o->slen[off + j] = bps[t][j + 1] - bps[t][j];
        }
        for (int j = 0; j <= nb; j++) o->spos[off + t + j] = bps[t][j];
        off += nb;
        free(bps[t]);
    }
    o->soff[nt] = off;
    free(bps);
    free(nbs);
    return 0;
}

/* ------------------------------------------------------------------------
 * z-stacks (Eq. 5) and the lattice coordinate zeta(s) = (z_0 + s cot)/dz.
 *
 * Reading of the unspecified axial laydown: per azimuth pair the polar angle
 * is corrected so that the cycle length times cot(theta) is a whole number of
 * axial spacings (cot' = c dz / L_cyc, c = max(1, round(L_cyc cot / dz))),
 * and z_0(T, theta) = dz/2 + S_T cot(theta) (mod dz) with S_T the start of T in
 * its cycle.  With S_T = M_T steps this is z_0/dz = frac(1/2 + M_T c / Mcyc),
 * an exact rational.  Every reflective link then lands on a track.
 * ---------------------------------------------------------------------- */

static void stack_geom(orc_t *o, int t, int p, long *zn, double *zf, int *nb_out,
                       double *cot_out, double *sin_out, double *cos_out) {
    int a = o->t_azim[t];
    int m = a < o->nq ? a : o->A / 2 - 1 - a;
    int ph = p % o->Ph, up = p < o->Ph;
    long c = o->cpol[m * o->Ph + ph], Mc = o->Mcyc[m];
    long r = up ? mod_l(Mc / 2 + (long)((__int128)o->t_M[t] * c % Mc), Mc)
                : mod_l(Mc / 2 - (long)((__int128)o->t_M[t] * c % Mc), Mc);
    double z0 = (double)r / (double)Mc;
    double cot = up ? o->cot[m * o->Ph + ph] : -o->cot[m * o->Ph + ph];
    double slope = (up ? 1.0 : -1.0) * (double)c / ((double)Mc * o->lu[m]); /* zeta per cm */
    long off = o->soff[t];
    int nb = (int)(o->soff[t + 1] - off);
    for (int j = 0; j <= nb; j++) {
        double s = o->spos[off + t + j];
        split_coord(o->pfrac, o->npfrac, z0 + s * slope, zn + j, zf + j);
    }
    *nb_out = nb;
    *cot_out = cot;
    *sin_out = o->sinp[m * o->Ph + ph];
    *cos_out = o->cosp[m * o->Ph + ph];
}

typedef struct {
    long imin;
    int ntrk;
    int *nseg;      /* per track */
    long *off;      /* per track + 1 */
    int *fsr;
    double *len;
    long cap_seg;
    int cap_trk;
    int *cursor;
    long *zn;       /* lattice coordinates at the 2D boundaries: integer parts */
    double *zf;     /* and fractional parts */
    int zcap;
} stackbuf;

static void sb_free(stackbuf *sb) {
    free(sb->nseg); free(sb->off); free(sb->fsr); free(sb->len); free(sb->cursor); free(sb->zn); free(sb->zf);
    memset(sb, 0, sizeof *sb);
}

/* Segments of every track of stack (t, p), collectively for the whole
 * z-stack (Sec. 2.2): per (2D segment b, layer L) the range of track indices
 * crossing it (Eqs. 6-7), classified by Eqs. 9-10.  All index arithmetic is
 * done in lattice units (z / dz) on split coordinates n + f (split_coord):
 * track i at boundary j lies at (i + zn[j]) + zf[j], a plane at
 * lplane[L] + qplane[L]. */
static void build_stack(orc_t *o, int t, int p, stackbuf *sb) {
    long off = o->soff[t];
    int nb = (int)(o->soff[t + 1] - off);
    if (sb->zcap < nb + 1) {
        free(sb->zn); free(sb->zf);
        sb->zcap = nb + 1;
        sb->zn = malloc(sizeof(long) * (size_t)sb->zcap);
        sb->zf = malloc(sizeof(double) * (size_t)sb->zcap);
    }
    double cot, sn, cs;
    int nbx;
    stack_geom(o, t, p, sb->zn, sb->zf, &nbx, &cot, &sn, &cs);
    const long *zn = sb->zn;
    const double *zf = sb->zf;
    int up = cot > 0;
    int NL = o->nl;
    /* track index range over the whole stack (domain 0 < u < Nz): the
       highest end above 0, the lowest below Nz */
    int e_hi = coord_lt(zn[0], zf[0], zn[nb], zf[nb]) ? nb : 0, e_lo = nb - e_hi;
    long imin = -zn[e_hi] + (zf[e_hi] > 0.0 ? 0 : 1);
    long imax = (long)o->Nz - 1 - zn[e_lo];
    int ntrk = (int)(imax - imin + 1);
    if (ntrk < 0) ntrk = 0;
    if (sb->cap_trk < ntrk) {
        free(sb->nseg); free(sb->off); free(sb->cursor);
        sb->cap_trk = ntrk;
        sb->nseg = malloc(sizeof(int) * (size_t)ntrk);
        sb->off = malloc(sizeof(long) * (size_t)(ntrk + 1));
        sb->cursor = malloc(sizeof(int) * (size_t)ntrk);
    }
    sb->imin = imin;
    sb->ntrk = ntrk;
    memset(sb->nseg, 0, sizeof(int) * (size_t)ntrk);
    for (int pass = 0; pass < 2; pass++) {
        if (pass == 1) {
            long tot = 0;
            for (int k = 0; k < ntrk; k++) { sb->off[k] = tot; tot += sb->nseg[k]; sb->cursor[k] = 0; }
            sb->off[ntrk] = tot;
            if (sb->cap_seg < tot) {
                free(sb->fsr); free(sb->len);
                sb->cap_seg = tot + 1024;
                sb->fsr = malloc(sizeof(int) * (size_t)sb->cap_seg);
                sb->len = malloc(sizeof(double) * (size_t)sb->cap_seg);
            }
        }
        for (int b = 0; b < nb; b++) {
            /* the segment's higher and lower end */
            int jh = coord_lt(zn[b], zf[b], zn[b + 1], zf[b + 1]) ? b + 1 : b, jl = 2 * b + 1 - jh;
            long nhi = zn[jh], nlo = zn[jl];
            double fhi = zf[jh], flo = zf[jl];
            int reg = o->sreg[off + b];
            double l2d = o->slen[off + b];
            for (int li = 0; li < NL; li++) {
                int L = up ? li : NL - 1 - li;     /* traversal order of the layers */
                long pmin = o->lplane[L], pmax = o->lplane[L + 1];
                double qmin = o->qplane[L], qmax = o->qplane[L + 1];
                /* Eq. 6: the smallest i with i + zhi >= kmin */
                long i_start = (pmin - nhi) + (qmin > fhi ? 1 : 0);
                /* Eq. 7: the largest i with i + zlo <= kmax */
                long i_end = (pmax - nlo) - (qmax >= flo ? 0 : 1);
                /* Eq. 9: the smallest i with i + zlo >= kmin */
                long i_in = (pmin - nlo) + (qmin > flo ? 1 : 0);
                /* Eq. 10: the largest i with i + zhi <= kmax */
                long i_out = (pmax - nhi) - (qmax >= fhi ? 0 : 1);
                if (i_start < imin) i_start = imin;
                if (i_end > imax) i_end = imax;
                for (long i = i_start; i <= i_end; i++) {
                    double len;
                    if (i >= i_in && i <= i_out) {
                        len = l2d / sn;                                                    /* Eq. 8 */
                    } else if (i_in > i_out && i > i_out && i < i_in) {
                        len = ((double)(pmax - pmin) + (qmax - qmin)) * o->dz / cs;         /* Eq. 11 */
                    } else {
                        /* a partial crossing; touching a plane only (zero
                           length) is no segment: i + zhi == kmin (i = i_start
                           with equal parts) or i + zlo == kmax (i = i_end) */
                        if ((i == pmin - nhi && qmin == fhi) || (i == pmax - nlo && qmax == flo))
                            continue;
                        /* the part inside the layer: from max(i + zlo, kmin)
                           to min(i + zhi, kmax) */
                        long an = i + nlo, bn = i + nhi;
                        double af = flo, bf = fhi;
                        if (coord_lt(an, af, pmin, qmin)) { an = pmin; af = qmin; }
                        if (coord_lt(pmax, qmax, bn, bf)) { bn = pmax; bf = qmax; }
                        double du = (double)(bn - an) + (bf - af);
                        if (du <= 0.0) continue;                                          /* (rounding) */
                        len = du * o->dz / cs;
                    }
                    int k = (int)(i - imin);
                    if (pass == 0) sb->nseg[k]++;
                    else {
                        long q = sb->off[k] + sb->cursor[k]++;
                        sb->fsr[q] = reg * NL + L;
                        sb->len[q] = len;
                    }
                }
            }
        }
    }
}

/* slot of track (t, p, i) or -1 if it does not exist */
static long slot_of(orc_t *o, int t, int p, long i) {
    long s = (long)t * o->P + p;
    long k = i - o->stk_imin[s];
    if (k < 0 || k >= o->stk_n[s]) return -1;
    return o->stk_slot[s] + k;
}

/* lattice coordinate of stack (t, p) at the start (end=0) or end (end=1) of t */
static double stack_zeta_end(orc_t *o, int t, int p, int end) {
    int a = o->t_azim[t];
    int m = a < o->nq ? a : o->A / 2 - 1 - a;
    int ph = p % o->Ph, up = p < o->Ph;
    long c = o->cpol[m * o->Ph + ph], Mc = o->Mcyc[m];
    long r = up ? mod_l(Mc / 2 + (long)((__int128)o->t_M[t] * c % Mc), Mc)
                : mod_l(Mc / 2 - (long)((__int128)o->t_M[t] * c % Mc), Mc);
    double z0 = (double)r / (double)Mc;
    if (!end) return snap(z0);
    double slope = (up ? 1.0 : -1.0) * (double)c / ((double)Mc * o->lu[m]);
    long off = o->soff[t];
    int nb = (int)(o->soff[t + 1] - off);
    return snap(z0 + o->spos[off + t + nb] * slope);
}

static long round_int(double x, int *ok) {
    double r = nearbyint(x);
    if (fabs(x - r) > 1e-6) *ok = 0;
    return (long)r;
}

/* Destination of the flux leaving track (t, p, i) in sense s (0 along t,
 * 1 against it), found geometrically from the exit point: reflect the
 * direction in the face it leaves by and find the track through that point.
 * An exit exactly on an edge between an axial and a radial face reflects in
 * both (the track reverses).  Vacuum faces give -1. */
static long link_dest(orc_t *o, int t, int p, long i, int s, int *ok) {
    int Ph = o->Ph, up = p < Ph;
    int pbar = up ? p + Ph : p - Ph;
    double zs = stack_zeta_end(o, t, p, 0), ze = stack_zeta_end(o, t, p, 1);
    double u = (double)i + (s == 0 ? ze : zs);   /* lattice height at the radial end of the exit */
    double Nz = (double)o->Nz;
    /* vertical direction of this traversal: +1 up, -1 down */
    int vert = (up ? 1 : -1) * (s == 0 ? 1 : -1);
    int axial_face = -1, radial = 0, corner = 0;
    if (vert > 0) {
        if (u < Nz) radial = 1;
        else if (u > Nz) axial_face = F_ZMAX;
        else { corner = 1; axial_face = F_ZMAX; }
    } else {
        if (u > 0.0) radial = 1;
        else if (u < 0.0) axial_face = F_ZMIN;
        else { corner = 1; axial_face = F_ZMIN; }
    }
    int rface = s == 0 ? o->t_eface[t] : o->t_sface[t];
    if (corner) {
        if (o->bc[axial_face] && o->bc[rface]) return slot_of(o, t, p, i) * 2 + (1 - s);
        return -1;
    }
    if (!radial) {
        if (!o->bc[axial_face]) return -1;
        double ub = axial_face == F_ZMAX ? Nz : 0.0;
        double zsb = stack_zeta_end(o, t, pbar, 0);
        long i2 = round_int(2.0 * ub - (double)i - (zs + zsb), ok);
        long sl = slot_of(o, t, pbar, i2);
        if (sl < 0) { *ok = 0; return -1; }
        return sl * 2 + s;
    }
    if (!o->bc[rface]) return -1;
    int t2 = o->succ_t[s][t], s2 = o->succ_s[s][t];
    /* the continuing traversal keeps the vertical direction */
    int q;
    if (s2 == 0) q = vert > 0 ? (p % Ph) : (p % Ph) + Ph;
    else q = vert > 0 ? (p % Ph) + Ph : (p % Ph);
    double zq = stack_zeta_end(o, t2, q, s2 == 0 ? 0 : 1);
    long i2 = round_int(u - zq, ok);
    long sl = slot_of(o, t2, q, i2);
    if (sl < 0) { *ok = 0; return -1; }
    return sl * 2 + s2;
}

/* ------------------------------------------------------------------------ */

void orc_destroy(void *h);

void *orc_create(const orc_input *in, char *err, int errlen) {
    if (!in || in->ncx < 1 || in->ncy < 1 || in->n_layers < 1 || in->G < 1 || in->M < 1 ||
        in->n_azim < 4 || in->n_azim % 4 || in->n_polar < 2 || in->n_polar % 2 ||
        !(in->radial_spacing > 0) || !(in->axial_spacing > 0) || !(in->pitch > 0) ||
        !(in->height > 0) || !(in->radius > 0) || 2 * in->radius >= in->pitch) {
        set_err(err, errlen, "invalid input");
        return NULL;
    }
    orc_t *o = calloc(1, sizeof(orc_t));
    o->ncx = in->ncx; o->ncy = in->ncy; o->nl = in->n_layers; o->M = in->M; o->G = in->G;
    o->A = in->n_azim; o->P = in->n_polar; o->pitch = in->pitch; o->radius = in->radius;
    o->H = in->height; o->nthreads = in->n_threads > 0 ? in->n_threads : 1;
    int nc = o->ncx * o->ncy, G = o->G, M = o->M;
    o->has_pin = malloc(sizeof(int) * (size_t)nc);
    memcpy(o->has_pin, in->has_pin, sizeof(int) * (size_t)nc);
    o->mat_in = malloc(sizeof(int) * (size_t)(nc * o->nl));
    o->mat_out = malloc(sizeof(int) * (size_t)(nc * o->nl));
    memcpy(o->mat_in, in->mat_in, sizeof(int) * (size_t)(nc * o->nl));
    memcpy(o->mat_out, in->mat_out, sizeof(int) * (size_t)(nc * o->nl));
    memcpy(o->bc, in->bc, sizeof o->bc);
    o->st = malloc(sizeof(double) * (size_t)(M * G));
    o->ss = malloc(sizeof(double) * (size_t)(M * G * G));
    o->nsf = malloc(sizeof(double) * (size_t)(M * G));
    o->chi = malloc(sizeof(double) * (size_t)(M * G));
    memcpy(o->st, in->sigma_t, sizeof(double) * (size_t)(M * G));
    memcpy(o->ss, in->sigma_s, sizeof(double) * (size_t)(M * G * G));
    memcpy(o->nsf, in->nu_sigma_f, sizeof(double) * (size_t)(M * G));
    memcpy(o->chi, in->chi, sizeof(double) * (size_t)(M * G));
    if (in->ext_source) {
        o->src = malloc(sizeof(double) * (size_t)(M * G));
        memcpy(o->src, in->ext_source, sizeof(double) * (size_t)(M * G));
    }
    for (int i = 0; i < M * G; i++) {
        if (!(o->st[i] > 0)) { set_err(err, errlen, "sigma_t must be positive"); orc_destroy(o); return NULL; }
    }
    o->Wx = o->ncx * o->pitch;
    o->Wy = o->ncy * o->pitch;
    /* pin-cell circles: the fuel circle split into rings of equal area
       (r_k^2 = r_f^2 k / F), then mod_rings circles whose squared radii step
       evenly from r_f^2 towards (pitch/2)^2 (that last circle excluded);
       sector s of S covers the angles [2 pi s / S, 2 pi (s + 1) / S) */
    if (in->fuel_rings < 0 || in->fuel_rings > 64 || in->mod_rings < 0 || in->mod_rings > 64 ||
        in->sectors < 0 || in->sectors > 64) {
        set_err(err, errlen, "rings and sectors must lie in [0, 64]");
        orc_destroy(o);
        return NULL;
    }
    o->nfuel_rings = in->fuel_rings > 0 ? in->fuel_rings : 1;
    o->nsec = in->sectors > 0 ? in->sectors : 1;
    o->ncirc = 0;
    for (int k = 1; k <= o->nfuel_rings; k++)
        o->circ_r2[o->ncirc++] = o->radius * o->radius * k / o->nfuel_rings;
    {
        double rf2 = o->radius * o->radius, rc2 = 0.25 * o->pitch * o->pitch;
        for (int k = 1; k <= in->mod_rings; k++)
            o->circ_r2[o->ncirc++] = rf2 + (rc2 - rf2) * k / (in->mod_rings + 1);
    }
    int per_pin = (o->ncirc + 1) * o->nsec;
    /* FSRs: radial regions cell by cell (pin cells: ring * sectors + sector,
       innermost ring first; other cells: one region), times layers */
    o->reg_base = malloc(sizeof(int) * (size_t)nc);
    int nr = 0;
    for (int c = 0; c < nc; c++) { o->reg_base[c] = nr; nr += o->has_pin[c] ? per_pin : 1; }
    o->nreg = nr;
    o->nfsr = nr * o->nl;
    o->fsr_mat = malloc(sizeof(int) * (size_t)o->nfsr);
    for (int c = 0; c < nc; c++) {
        for (int L = 0; L < o->nl; L++) {
            if (o->has_pin[c]) {
                for (int ring = 0; ring <= o->ncirc; ring++)
                    for (int s = 0; s < o->nsec; s++)
                        o->fsr_mat[(o->reg_base[c] + ring * o->nsec + s) * o->nl + L] =
                            ring < o->nfuel_rings ? o->mat_in[c * o->nl + L] : o->mat_out[c * o->nl + L];
            } else {
                o->fsr_mat[o->reg_base[c] * o->nl + L] = o->mat_out[c * o->nl + L];
            }
        }
    }
    for (int i = 0; i < o->nfsr; i++)
        if (o->fsr_mat[i] < 0 || o->fsr_mat[i] >= M) { set_err(err, errlen, "material index out of range"); orc_destroy(o); return NULL; }
    /* axial lattice: dz_eff = H / Nz.  Equal layers of cpl lattice cells
       each when the height divides; otherwise layer planes in lattice units,
       anywhere (the local axial mesh of Sec. 2.2), with exact plane ties
       (split_coord) */
    double q = o->H / in->axial_spacing;
    long Nz = (fabs(q - nearbyint(q)) < 1e-9) ? (long)nearbyint(q) : (long)ceil(q);
    o->Nz = (int)Nz;
    o->dz = o->H / (double)Nz;
    o->lplane = malloc(sizeof(long) * (size_t)(o->nl + 1));
    o->kplane = malloc(sizeof(double) * (size_t)(o->nl + 1));
    o->qplane = malloc(sizeof(double) * (size_t)(o->nl + 1));
    o->pfrac = malloc(sizeof(double) * (size_t)(o->nl + 1));
    o->npfrac = 0;
    if (!in->layer_z && Nz % o->nl == 0) {
        o->cpl = (int)(Nz / o->nl);
        for (int L = 0; L <= o->nl; L++) {
            o->lplane[L] = (long)L * o->cpl;
            o->kplane[L] = (double)o->lplane[L];
            o->qplane[L] = 0.0;
        }
    } else {
        /* planes in lattice units (equal layers off the lattice: the planes
           L H / n_layers); a plane within 1e-9 of a lattice index is that
           index; the first is 0 and the last the height, increasing */
        o->cpl = 0;
        for (int L = 0; L <= o->nl; L++) {
            double zl = in->layer_z ? in->layer_z[L] : (double)L * o->H / (double)o->nl;
            double u = zl / o->dz;
            double k = nearbyint(u);
            if (fabs(u - k) <= 1e-9) u = k;
            if ((L == 0 && u != 0.0) || (L == o->nl && u != (double)Nz) ||
                (L > 0 && !(u > o->kplane[L - 1] + 1e-6)) || !isfinite(u)) {
                set_err(err, errlen, "layer planes must rise from 0 to the height");
                orc_destroy(o);
                return NULL;
            }
            o->kplane[L] = u;
            o->lplane[L] = (long)floor(u);
        }
        /* distinct fractional parts of the interior planes, ascending */
        for (int L = 1; L < o->nl; L++) {
            double f = o->kplane[L] - floor(o->kplane[L]);
            if (f == 0.0) continue;
            int seen = 0;
            for (int q = 0; q < o->npfrac; q++) seen |= fabs(o->pfrac[q] - f) <= TIE_EPS;
            if (!seen) o->pfrac[o->npfrac++] = f;
        }
        for (int a = 1; a < o->npfrac; a++)
            for (int b = a; b > 0 && o->pfrac[b - 1] > o->pfrac[b]; b--) {
                double t = o->pfrac[b]; o->pfrac[b] = o->pfrac[b - 1]; o->pfrac[b - 1] = t;
            }
        /* each plane's fraction is its pfrac entry (planes whose fractions
           tie within TIE_EPS share one) */
        for (int L = 0; L <= o->nl; L++) {
            long n;
            double f;
            split_coord(o->pfrac, o->npfrac, o->kplane[L], &n, &f);
            o->lplane[L] = n;
            o->qplane[L] = f;
        }
    }
    /* azimuths */
    o->nq = o->A / 4;
    int nq = o->nq;
    o->nx = calloc(nq, sizeof(long)); o->ny = calloc(nq, sizeof(long));
    o->gg = calloc(nq, sizeof(long)); o->Mcyc = calloc(nq, sizeof(long));
    o->phi_eff = calloc(nq, sizeof(double)); o->span = calloc(nq, sizeof(double));
    o->deff = calloc(nq, sizeof(double)); o->lu = calloc(nq, sizeof(double));
    for (int m = 0; m < nq; m++) {
        double phi = 2.0 * ORC_PI * (m + 0.5) / o->A;
        o->nx[m] = (long)ceil(o->Wx * fabs(sin(phi)) / in->radial_spacing);
        o->ny[m] = (long)ceil(o->Wy * fabs(cos(phi)) / in->radial_spacing);
        o->phi_eff[m] = atan2(o->Wy * o->nx[m], o->Wx * o->ny[m]);
        o->deff[m] = (o->Wx / o->nx[m]) * sin(o->phi_eff[m]);
        o->gg[m] = gcd_l(o->nx[m], o->ny[m]);
        o->Mcyc[m] = 4 * o->nx[m] * o->ny[m] / o->gg[m];
        double ux = o->Wx / (2.0 * o->nx[m]), uy = o->Wy / (2.0 * o->ny[m]);
        o->lu[m] = sqrt(ux * ux + uy * uy);
    }
    for (int m = 0; m < nq; m++) {
        double lo = m == 0 ? -o->phi_eff[0] : o->phi_eff[m - 1];
        double hi = m == nq - 1 ? ORC_PI - o->phi_eff[nq - 1] : o->phi_eff[m + 1];
        o->span[m] = 0.5 * (hi - lo);
    }
    /* polar: Gauss-Legendre in mu on (0, 1), Ph per hemisphere */
    o->Ph = o->P / 2;
    int Ph = o->Ph;
    double *x = malloc(sizeof(double) * Ph), *w = malloc(sizeof(double) * Ph);
    gauss_legendre(Ph, x, w);
    o->mu_gl = malloc(sizeof(double) * Ph);
    o->w_gl = malloc(sizeof(double) * Ph);
    for (int j = 0; j < Ph; j++) { /* ascending mu */
        o->mu_gl[j] = 0.5 * (1.0 + x[Ph - 1 - j]);
        o->w_gl[j] = 0.5 * w[Ph - 1 - j];
    }
    free(x); free(w);
    o->cpol = malloc(sizeof(long) * (size_t)(nq * Ph));
    o->cot = malloc(sizeof(double) * (size_t)(nq * Ph));
    o->sinp = malloc(sizeof(double) * (size_t)(nq * Ph));
    o->cosp = malloc(sizeof(double) * (size_t)(nq * Ph));
    o->W = malloc(sizeof(double) * (size_t)(nq * Ph));
    for (int m = 0; m < nq; m++) {
        double Lc = (double)o->Mcyc[m] * o->lu[m];
        for (int j = 0; j < Ph; j++) {
            double mu = o->mu_gl[j];
            double cot0 = mu / sqrt(1.0 - mu * mu);
            long c = (long)nearbyint(Lc * cot0 / o->dz);
            if (c < 1) c = 1;
            double cot = (double)c * o->dz / Lc;
            double sn = 1.0 / sqrt(1.0 + cot * cot);
            o->cpol[m * Ph + j] = c;
            o->cot[m * Ph + j] = cot;
            o->sinp[m * Ph + j] = sn;
            o->cosp[m * Ph + j] = cot * sn;
            /* track weight: azimuthal span x polar weight x cross-section area */
            o->W[m * Ph + j] = o->span[m] * o->w_gl[j] * o->deff[m] * o->dz * sn;
        }
    }
    if (build_2d(o, err, errlen)) { orc_destroy(o); return NULL; }
    build_2d_segments(o);
    /* stacks: index ranges and slots */
    long nstk = (long)o->nt * o->P;
    o->stk_imin = malloc(sizeof(long) * (size_t)nstk);
    o->stk_n = malloc(sizeof(long) * (size_t)nstk);
    o->stk_slot = malloc(sizeof(long) * (size_t)(nstk + 1));
    long slot = 0;
    for (int t = 0; t < o->nt; t++) {
        for (int p = 0; p < o->P; p++) {
            double zs = stack_zeta_end(o, t, p, 0), ze = stack_zeta_end(o, t, p, 1);
            double zmx = zs > ze ? zs : ze, zmn = zs < ze ? zs : ze;
            long imin = (long)floor(-zmx) + 1;
            long imax = (long)ceil((double)o->Nz - zmn) - 1;
            long s = (long)t * o->P + p;
            o->stk_imin[s] = imin;
            o->stk_n[s] = imax >= imin ? imax - imin + 1 : 0;
            o->stk_slot[s] = slot;
            slot += o->stk_n[s];
        }
    }
    o->stk_slot[nstk] = slot;
    o->n3d = slot;
    if (in->light) {
        o->phi = calloc((size_t)o->nfsr * G, sizeof(double));
        return o;  /* stacks and segments only: orc_stack, orc_sweep_sample */
    }
    o->dest = malloc(sizeof(long) * (size_t)(2 * o->n3d));
    int ok = 1;
    for (int t = 0; t < o->nt; t++)
        for (int p = 0; p < o->P; p++) {
            long s = (long)t * o->P + p;
            for (long k = 0; k < o->stk_n[s]; k++)
                for (int sense = 0; sense < 2; sense++)
                    o->dest[(o->stk_slot[s] + k) * 2 + sense] = link_dest(o, t, p, o->stk_imin[s] + k, sense, &ok);
        }
    if (!ok) { set_err(err, errlen, "3D link did not land on a track"); orc_destroy(o); return NULL; }
    /* state */
    o->V = calloc((size_t)o->nfsr, sizeof(double));
    o->phi = calloc((size_t)o->nfsr * G, sizeof(double));
    o->fiss_old = calloc((size_t)o->nfsr, sizeof(double));
    o->psi0 = calloc((size_t)o->n3d * 2 * G, sizeof(double));
    o->psi1 = calloc((size_t)o->n3d * 2 * G, sizeof(double));
    /* tracked volumes: V_i = sum over directions of (w/4pi) sum dA * len; each
     * stored track carries two directions of equal weight */
    stackbuf sb;
    memset(&sb, 0, sizeof sb);
    for (int t = 0; t < o->nt; t++) {
        int a = o->t_azim[t];
        int m = a < o->nq ? a : o->A / 2 - 1 - a;
        for (int p = 0; p < o->P; p++) {
            build_stack(o, t, p, &sb);
            double Wt = o->W[m * Ph + p % Ph];
            for (long qq = 0; qq < sb.off[sb.ntrk]; qq++)
                o->V[sb.fsr[qq]] += 2.0 * Wt * sb.len[qq] / (4.0 * ORC_PI);
        }
    }
    sb_free(&sb);
    return o;
}

void orc_destroy(void *h) {
    orc_t *o = (orc_t *)h;
    if (!o) return;
    void *ptrs[] = {o->lplane, o->kplane, o->qplane, o->pfrac, o->has_pin, o->mat_in, o->mat_out, o->st, o->ss, o->nsf, o->chi, o->src,
                    o->reg_base, o->fsr_mat, o->nx, o->ny, o->gg, o->Mcyc, o->phi_eff, o->span,
                    o->deff, o->lu, o->mu_gl, o->w_gl, o->cpol, o->cot, o->sinp, o->cosp,
                    o->a_off, o->t_azim, o->t_sface, o->t_sk, o->t_eface, o->t_ek, o->t_steps,
                    o->t_M, o->t_x0, o->t_y0, o->t_len, o->succ_t[0], o->succ_t[1],
                    o->succ_s[0], o->succ_s[1], o->soff, o->sreg, o->slen, o->spos,
                    o->stk_imin, o->stk_n, o->stk_slot, o->dest, o->W, o->V, o->phi, o->psi0,
                    o->psi1, o->fiss_old, o->start_tab, o->end_tab};
    for (size_t i = 0; i < sizeof ptrs / sizeof ptrs[0]; i++) free(ptrs[i]);
    free(o);
}

/* ------------------------------------------------------------------------
 * queries used by the tests
 * ---------------------------------------------------------------------- */

int orc_counts(void *h, int64_t *out) {
    orc_t *o = (orc_t *)h;
    out[0] = o->nfsr; out[1] = o->nreg; out[2] = o->nt; out[3] = (int64_t)o->nt * o->P;
    out[4] = o->n3d; out[5] = o->soff[o->nt]; out[6] = o->nq; out[7] = o->Ph;
    out[8] = o->Nz; out[9] = o->cpl;
    return 0;
}

/* out: nx, ny, gcd, Mcyc, phi_eff, delta_eff, span, step length */
int orc_azimuth(void *h, int m, double *out) {
    orc_t *o = (orc_t *)h;
    if (m < 0 || m >= o->nq) return -1;
    out[0] = (double)o->nx[m]; out[1] = (double)o->ny[m]; out[2] = (double)o->gg[m];
    out[3] = (double)o->Mcyc[m]; out[4] = o->phi_eff[m]; out[5] = o->deff[m];
    out[6] = o->span[m]; out[7] = o->lu[m];
    return 0;
}

/* out: c, cot, sin, cos, weight, mu_gl, w_gl, track weight W */
int orc_polar(void *h, int m, int ph, double *out) {
    orc_t *o = (orc_t *)h;
    if (m < 0 || m >= o->nq || ph < 0 || ph >= o->Ph) return -1;
    int i = m * o->Ph + ph;
    out[0] = (double)o->cpol[i]; out[1] = o->cot[i]; out[2] = o->sinp[i]; out[3] = o->cosp[i];
    out[4] = o->w_gl[ph]; out[5] = o->mu_gl[ph]; out[6] = o->w_gl[ph]; out[7] = o->W[i];
    return 0;
}

/* out: azim, sface, sk, eface, ek, steps, M, x0, y0, len, succ_t0, succ_s0, succ_t1, succ_s1, nseg */
int orc_track2d(void *h, int t, double *out) {
    orc_t *o = (orc_t *)h;
    if (t < 0 || t >= o->nt) return -1;
    out[0] = o->t_azim[t]; out[1] = o->t_sface[t]; out[2] = o->t_sk[t]; out[3] = o->t_eface[t];
    out[4] = o->t_ek[t]; out[5] = (double)o->t_steps[t]; out[6] = (double)o->t_M[t];
    out[7] = o->t_x0[t]; out[8] = o->t_y0[t]; out[9] = o->t_len[t];
    out[10] = o->succ_t[0][t]; out[11] = o->succ_s[0][t]; out[12] = o->succ_t[1][t];
    out[13] = o->succ_s[1][t]; out[14] = (double)(o->soff[t + 1] - o->soff[t]);
    return 0;
}

int orc_segments2d(void *h, int t, int *reg, double *len, double *pos) {
    orc_t *o = (orc_t *)h;
    if (t < 0 || t >= o->nt) return -1;
    long off = o->soff[t];
    int nb = (int)(o->soff[t + 1] - off);
    for (int j = 0; j < nb; j++) { reg[j] = o->sreg[off + j]; len[j] = o->slen[off + j]; }
    if (pos) for (int j = 0; j <= nb; j++) pos[j] = o->spos[off + t + j];
    return nb;
}

/* lattice coordinates zeta_j of stack (t, p) at the 2D boundaries */
int orc_stack_zeta(void *h, int t, int p, double *zeta) {
    orc_t *o = (orc_t *)h;
    if (t < 0 || t >= o->nt || p < 0 || p >= o->P) return -1;
    double cot, sn, cs;
    int nb = (int)(o->soff[t + 1] - o->soff[t]);
    long *zn = malloc(sizeof(long) * (size_t)(nb + 1));
    double *zf = malloc(sizeof(double) * (size_t)(nb + 1));
    stack_geom(o, t, p, zn, zf, &nb, &cot, &sn, &cs);
    for (int j = 0; j <= nb; j++) zeta[j] = (double)zn[j] + zf[j];
    free(zn);
    free(zf);
    return nb;
}

/* Segments of stack (t, p).  out_i[k]: track index i of the k-th listed track,
 * nseg[k]: its segment count; fsr/len concatenated in traversal order along t.
 * Only tracks with at least one segment are listed.  Returns the number of
 * tracks, or -(needed) if a capacity is too small. */
int64_t orc_stack(void *h, int t, int p, int64_t cap_trk, int64_t cap_seg, int64_t *out_i,
                  int32_t *nseg, int32_t *fsr, double *len, int64_t *nseg_total) {
    orc_t *o = (orc_t *)h;
    if (t < 0 || t >= o->nt || p < 0 || p >= o->P) return 0;
    stackbuf sb;
    memset(&sb, 0, sizeof sb);
    build_stack(o, t, p, &sb);
    long tot = sb.off[sb.ntrk];
    int ntr = 0;
    for (int k = 0; k < sb.ntrk; k++) if (sb.nseg[k]) ntr++;
    *nseg_total = tot;
    if (ntr > cap_trk || tot > cap_seg) { sb_free(&sb); return -1; }
    int q = 0;
    for (int k = 0; k < sb.ntrk; k++) {
        if (!sb.nseg[k]) continue;
        out_i[q] = sb.imin + k;
        nseg[q] = sb.nseg[k];
        q++;
    }
    for (long j = 0; j < tot; j++) { fsr[j] = sb.fsr[j]; len[j] = sb.len[j]; }
    sb_free(&sb);
    return ntr;
}

/* stack index range: out = imin, n */
int orc_stack_range(void *h, int t, int p, int64_t *out) {
    orc_t *o = (orc_t *)h;
    long s = (long)t * o->P + p;
    out[0] = o->stk_imin[s];
    out[1] = o->stk_n[s];
    return 0;
}

/* destination of (t, p, i, sense): out = t2, p2, i2, sense2 (all -1 if it leaks) */
int orc_link(void *h, int t, int p, int64_t i, int sense, int64_t *out) {
    orc_t *o = (orc_t *)h;
    if (!o->dest) return -1;
    long sl = slot_of(o, t, p, i);
    if (sl < 0) return -1;
    long d = o->dest[sl * 2 + sense];
    if (d < 0) { out[0] = out[1] = out[2] = out[3] = -1; return 0; }
    long dsl = d / 2;
    /* invert the slot numbering */
    long lo = 0, hi = (long)o->nt * o->P - 1;
    while (lo < hi) {
        long mid = (lo + hi + 1) / 2;
        if (o->stk_slot[mid] <= dsl) lo = mid; else hi = mid - 1;
    }
    while (lo + 1 < (long)o->nt * o->P && o->stk_slot[lo + 1] <= dsl && o->stk_n[lo] == 0) lo++;
    out[0] = lo / o->P; out[1] = lo % o->P;
    out[2] = o->stk_imin[lo] + (dsl - o->stk_slot[lo]);
    out[3] = d % 2;
    return 0;
}

int orc_volumes(void *h, double *V) {
    orc_t *o = (orc_t *)h;
    if (!o->V) return -1;
    memcpy(V, o->V, sizeof(double) * (size_t)o->nfsr);
    return 0;
}

int orc_fsr_materials(void *h, int32_t *mat) {
    orc_t *o = (orc_t *)h;
    for (int i = 0; i < o->nfsr; i++) mat[i] = o->fsr_mat[i];
    return 0;
}

/* ------------------------------------------------------------------------
 * transport sweep (Alg. 1 order, Eq. 3 per segment, tally per Eq. 4)
 * ---------------------------------------------------------------------- */

static void sweep(orc_t *o, const double *Q, double *tally, double *leak_out) {
    int G = o->G, Ph = o->Ph, nt = o->nt, P = o->P;
    int nth = o->nthreads;
    double *tl = calloc((size_t)nth * o->nfsr * G, sizeof(double));
    double *lk = calloc((size_t)nth, sizeof(double));
    double *psi_in = o->psi0, *psi_out = o->psi1;
    memset(psi_out, 0, sizeof(double) * (size_t)o->n3d * 2 * G);
#pragma omp parallel num_threads(nth)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = tl + (size_t)tid * o->nfsr * G;
        double *psi = malloc(sizeof(double) * (size_t)G);
        stackbuf sb;
        memset(&sb, 0, sizeof sb);
#pragma omp for schedule(static)
        for (int t = 0; t < nt; t++) {                       /* for each 2D track   */
            int a = o->t_azim[t];
            int m = a < o->nq ? a : o->A / 2 - 1 - a;
            for (int p = 0; p < P; p++) {                    /* for each polar angle */
                build_stack(o, t, p, &sb);                   /* getTrackOTF + traceSegmentsOTF */
                double Wt = o->W[m * Ph + p % Ph];
                long s = (long)t * P + p;
                for (int k = 0; k < sb.ntrk; k++) {          /* for each z in stack  */
                    long i = sb.imin + k;
                    long kk = i - o->stk_imin[s];
                    if (kk < 0 || kk >= o->stk_n[s]) continue;
                    long sl = o->stk_slot[s] + kk;
                    long b0 = sb.off[k], n = sb.nseg[k];
                    for (int sense = 0; sense < 2; sense++) { /* transportsweep */
                        for (int g = 0; g < G; g++) psi[g] = psi_in[(sl * 2 + sense) * G + g];
                        for (long j = 0; j < n; j++) {
                            long q = sense == 0 ? b0 + j : b0 + n - 1 - j;
                            int f = sb.fsr[q];
                            const double *sig = o->st + (size_t)o->fsr_mat[f] * G;
                            for (int g = 0; g < G; g++) {
                                double e = exp(-sig[g] * sb.len[q]);
                                double qs = Q[(size_t)f * G + g] / sig[g];
                                double out = psi[g] * e + qs * (1.0 - e);   /* Eq. 3 */
                                my[(size_t)f * G + g] += Wt * (psi[g] - out);
                                psi[g] = out;
                            }
                        }
                        long d = o->dest[sl * 2 + sense];
                        if (d >= 0) {
                            for (int g = 0; g < G; g++) psi_out[d * G + g] = psi[g];
                        } else {
                            for (int g = 0; g < G; g++) lk[tid] += Wt * psi[g];
                        }
                    }
                }
            }
        }
        free(psi);
        sb_free(&sb);
    }
    memset(tally, 0, sizeof(double) * (size_t)o->nfsr * G);
    double leak = 0.0;
    for (int th = 0; th < nth; th++) {
        const double *my = tl + (size_t)th * o->nfsr * G;
        for (size_t q = 0; q < (size_t)o->nfsr * G; q++) tally[q] += my[q];
        leak += lk[th];
    }
    *leak_out = leak;
    free(tl);
    free(lk);
    /* Jacobi boundary fluxes: this sweep's outgoing fluxes feed the next one */
    double *tmp = o->psi0; o->psi0 = o->psi1; o->psi1 = tmp;
}

/* isotropic source per steradian: Q = (scatter + chi/k fission + S) / 4 pi */
static void source(orc_t *o, const double *phi, double k, double *Q) {
    int G = o->G;
    for (int i = 0; i < o->nfsr; i++) {
        int m = o->fsr_mat[i];
        const double *ph = phi + (size_t)i * G;
        double fis = 0.0;
        for (int h = 0; h < G; h++) fis += o->nsf[m * G + h] * ph[h];
        for (int g = 0; g < G; g++) {
            double sc = 0.0;
            for (int h = 0; h < G; h++) sc += o->ss[(m * G + h) * G + g] * ph[h];
            double q = sc + o->chi[m * G + g] * fis / k;
            if (o->src) q += o->src[m * G + g];
            Q[(size_t)i * G + g] = q / (4.0 * ORC_PI);
        }
    }
}

static double production(orc_t *o, const double *phi) {
    double P = 0.0;
    int G = o->G;
    for (int i = 0; i < o->nfsr; i++) {
        int m = o->fsr_mat[i];
        for (int g = 0; g < G; g++) P += o->V[i] * o->nsf[m * G + g] * phi[(size_t)i * G + g];
    }
    return P;
}

static double absorption(orc_t *o, const double *phi) {
    double Ab = 0.0;
    int G = o->G;
    for (int i = 0; i < o->nfsr; i++) {
        int m = o->fsr_mat[i];
        for (int g = 0; g < G; g++) {
            double sa = o->st[m * G + g];
            for (int h = 0; h < G; h++) sa -= o->ss[(m * G + g) * G + h];
            Ab += o->V[i] * sa * phi[(size_t)i * G + g];
        }
    }
    return Ab;
}

int orc_set_threads(void *h, int n) { ((orc_t *)h)->nthreads = n > 0 ? n : 1; return 0; }

/* initial state: phi = 1, boundary fluxes 0, k = 1 (fission source normalised
 * to one for eigenvalue problems) */
int orc_reset(void *h) {
    orc_t *o = (orc_t *)h;
    if (!o->psi0) return -1;
    size_t n = (size_t)o->nfsr * o->G;
    for (size_t q = 0; q < n; q++) o->phi[q] = 1.0;
    memset(o->psi0, 0, sizeof(double) * (size_t)o->n3d * 2 * o->G);
    memset(o->psi1, 0, sizeof(double) * (size_t)o->n3d * 2 * o->G);
    o->k = 1.0;
    if (!o->src) {
        double P = production(o, o->phi);
        if (P > 0) for (size_t q = 0; q < n; q++) o->phi[q] /= P;
    }
    int G = o->G;
    for (int i = 0; i < o->nfsr; i++) {
        double f = 0.0;
        int m = o->fsr_mat[i];
        for (int g = 0; g < G; g++) f += o->nsf[m * G + g] * o->phi[(size_t)i * G + g];
        o->fiss_old[i] = f;
    }
    return 0;
}

/* Power (or fixed-source) iteration.  out: k, iterations, residual,
 * production, absorption, leakage, converged, dk.  max_iter iterations at
 * most; stops when |dk| < tol_k and the residual < tol_src (tol_k ignored for
 * fixed-source problems).  tol_src <= 0 runs exactly max_iter iterations. */
int orc_iterate(void *h, int max_iter, double tol_k, double tol_src, double *out) {
    orc_t *o = (orc_t *)h;
    if (!o->psi0) return -1;
    int G = o->G;
    size_t n = (size_t)o->nfsr * G;
    double *Q = malloc(sizeof(double) * n), *tally = malloc(sizeof(double) * n);
    double *phin = malloc(sizeof(double) * n);
    int eig = o->src == NULL;
    int it = 0, conv = 0;
    double res = 0.0, dk = 0.0, leak = 0.0;
    for (it = 0; it < max_iter;) {
        source(o, o->phi, o->k, Q);
        sweep(o, Q, tally, &leak);
        for (int i = 0; i < o->nfsr; i++) {
            int m = o->fsr_mat[i];
            for (int g = 0; g < G; g++) {
                size_t q = (size_t)i * G + g;
                double tv = o->V[i] > 0 ? tally[q] / o->V[i] : 0.0;
                phin[q] = (4.0 * ORC_PI * Q[q] + tv) / o->st[m * G + g];
            }
        }
        double knew = o->k;
        if (eig) {
            double Pn = production(o, phin);
            knew = o->k * Pn;   /* previous flux was normalised to P = 1 */
            for (size_t q = 0; q < n; q++) phin[q] /= Pn;
            for (size_t q = 0; q < (size_t)o->n3d * 2 * G; q++) o->psi0[q] /= Pn;
            leak /= Pn;
            double acc = 0.0;
            int cnt = 0;
            for (int i = 0; i < o->nfsr; i++) {
                int m = o->fsr_mat[i];
                double f = 0.0;
                for (int g = 0; g < G; g++) f += o->nsf[m * G + g] * phin[(size_t)i * G + g];
                if (f > 0) { double r = (f - o->fiss_old[i]) / f; acc += r * r; cnt++; }
                o->fiss_old[i] = f;
            }
            res = cnt ? sqrt(acc / cnt) : 0.0;
        } else {
            double acc = 0.0;
            int cnt = 0;
            for (size_t q = 0; q < n; q++)
                if (phin[q] > 0) { double r = (phin[q] - o->phi[q]) / phin[q]; acc += r * r; cnt++; }
            res = cnt ? sqrt(acc / cnt) : 0.0;
        }
        dk = knew - o->k;
        o->k = knew;
        memcpy(o->phi, phin, sizeof(double) * n);
        it++;
        if (tol_src > 0 && res < tol_src && (!eig || fabs(dk) < tol_k)) { conv = 1; break; }
    }
    o->last_leak = leak;
    o->last_res = res;
    out[0] = o->k; out[1] = it; out[2] = res; out[3] = production(o, o->phi);
    out[4] = absorption(o, o->phi); out[5] = leak; out[6] = conv; out[7] = dk;
    free(Q); free(tally); free(phin);
    return 0;
}

int orc_get_flux(void *h, double *phi) {
    orc_t *o = (orc_t *)h;
    memcpy(phi, o->phi, sizeof(double) * (size_t)o->nfsr * o->G);
    return 0;
}

int orc_set_flux(void *h, const double *phi, double k) {
    orc_t *o = (orc_t *)h;
    memcpy(o->phi, phi, sizeof(double) * (size_t)o->nfsr * o->G);
    o->k = k;
    return 0;
}

/* One sweep from a given source Q (per steradian, [nfsr*G]) with the current
 * boundary fluxes; returns the tally and leakage and advances the boundary
 * fluxes.  Used for sampled single-sweep parity and CPU timing. */
int orc_sweep_once(void *h, const double *Q, double *tally, double *leak) {
    orc_t *o = (orc_t *)h;
    if (!o->psi0) return -1;
    sweep(o, Q, tally, leak);
    return 0;
}

/* Sweep only the 2D tracks in [t0, t1) (all polar angles), from source Q,
 * with zero incoming fluxes: a bounded sample of the sweep for CPU timing.
 * Returns the number of segment-group integrations performed. */
int64_t orc_sweep_sample(void *h, const double *Q, int t0, int t1, double *tally) {
    orc_t *o = (orc_t *)h;
    int G = o->G, Ph = o->Ph, P = o->P;
    int nth = o->nthreads;
    int64_t total = 0;
    double *tl = calloc((size_t)nth * o->nfsr * G, sizeof(double));
#pragma omp parallel num_threads(nth) reduction(+ : total)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *my = tl + (size_t)tid * o->nfsr * G;
        double *psi = malloc(sizeof(double) * (size_t)G);
        stackbuf sb;
        memset(&sb, 0, sizeof sb);
#pragma omp for schedule(static)
        for (int t = t0; t < t1; t++) {
            int a = o->t_azim[t];
            int m = a < o->nq ? a : o->A / 2 - 1 - a;
            for (int p = 0; p < P; p++) {
                build_stack(o, t, p, &sb);
                double Wt = o->W[m * Ph + p % Ph];
                for (int k = 0; k < sb.ntrk; k++) {
                    long b0 = sb.off[k], n = sb.nseg[k];
                    for (int sense = 0; sense < 2; sense++) {
                        for (int g = 0; g < G; g++) psi[g] = 0.0;
                        for (long j = 0; j < n; j++) {
                            long q = sense == 0 ? b0 + j : b0 + n - 1 - j;
                            int f = sb.fsr[q];
                            const double *sig = o->st + (size_t)o->fsr_mat[f] * G;
                            for (int g = 0; g < G; g++) {
                                double e = exp(-sig[g] * sb.len[q]);
                                double qs = Q[(size_t)f * G + g] / sig[g];
                                double out = psi[g] * e + qs * (1.0 - e);
                                my[(size_t)f * G + g] += Wt * (psi[g] - out);
                                psi[g] = out;
                            }
                        }
                        total += n * G;
                    }
                }
            }
        }
        free(psi);
        sb_free(&sb);
    }
    memset(tally, 0, sizeof(double) * (size_t)o->nfsr * G);
    for (int th = 0; th < nth; th++)
        for (size_t q = 0; q < (size_t)o->nfsr * G; q++) tally[q] += tl[(size_t)th * o->nfsr * G + q];
    free(tl);
    return total;
}

/* boundary flux of one (t, p, i, sense) slot: the incoming flux of the next
 * sweep for that track and direction */
int orc_psi(void *h, int t, int p, int64_t i, int sense, double *val, int set) {
    orc_t *o = (orc_t *)h;
    if (!o->psi0) return -1;
    long sl = slot_of(o, t, p, i);
    if (sl < 0) return -1;
    double *ps = o->psi0 + (sl * 2 + sense) * o->G;
    for (int g = 0; g < o->G; g++) {
        if (set) ps[g] = val[g]; else val[g] = ps[g];
    }
    return 0;
}

int orc_clear_psi(void *h) {
    orc_t *o = (orc_t *)h;
    if (!o->psi0) return -1;
    memset(o->psi0, 0, sizeof(double) * (size_t)o->n3d * 2 * o->G);
    return 0;
}
