/*
 * fsl_oracle.c -- plain, slow, FP64 CPU oracle of one free-surface lattice
 * Boltzmann (FSLBM) time step with finite-difference (FD) and least-squares
 * (LSQR) curvature, after Bogner, Ruede, Harting, arXiv 1509.07691.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA path; the two meet only in the byte
 * layout of the arrays they exchange (D3Q19 order, flag bits, SoA index).
 *
 * Every loop runs over whole arrays in index order; nothing is blocked, fused
 * or reordered beyond what the equations state.  Each function names the part
 * of the paper it follows.  Where the paper is silent the reading taken is
 * stated in place.  Parity status (what pins each function) is recorded in the
 * header comment of each exported function.
 *
 * Conventions
 *   cell index   i = x + nx*(y + ny*z); all three axes wrap periodically;
 *                walls are OBSTACLE cells in the grid.
 *   PDF layout   f[q*N + i], q in the D3Q19 order below.
 *   flags        1 = liquid, 2 = interface, 4 = gas, 8 = obstacle.
 *   normals      n points towards the liquid (n = grad phi, Sec. II.A).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NQ 19
/* D3Q19 lattice velocities (Sec. II): rest, 6 faces, 12 edges; q and its
 * opposite are neighbours in this order (1<->2, 3<->4, ...). */
static const int CXQ[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CYQ[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZQ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

#define FL_LIQ 1
#define FL_IF 2
#define FL_GAS 4
#define FL_OBS 8
#define FL_TYPE 15

typedef struct {
    int nx, ny, nz;
    int collision;   /* 0 = BGK, 1 = TRT (Sec. II) */
    int curv_model;  /* 0 = LSQR (Sec. II.C), 1 = FD (Sec. II.A), 2 = none (kappa = 0),
                        4 = TR (Sec. II.B) */
    int literal_phi; /* 1 = update phi by Eq. (advection1) literally instead of tracking mass */
    double tau;      /* relaxation time, nu = (tau - 1/2)/3 */
    double magic;    /* TRT parameter Lambda = (tau_e - 1/2)(tau_o - 1/2) */
    double sigma;    /* surface tension */
    double p_gas;    /* gas pressure p_g */
    double theta;    /* equilibrium contact angle theta_eq in radians */
    double eps;      /* conversion threshold */
    int frozen;      /* 1 = cell types frozen: no conversion test, no excess mass */
    int excess_rule; /* 0 = equal shares (reading O7), 1 = normal-weighted shares (reading K1) */
} orc_params;

typedef struct {
    int kind;        /* 0 sphere, 1 P2-perturbed sphere, 2 spherical cap above z = zw,
                        3 two spheres, 4 sinusoidal pool, 5 half-space */
    int invert;      /* 1: liquid outside the shape (a bubble) */
    int sub;         /* sub-samples per axis */
    int pad_;
    double c[3], R, eps2;
    double c2[3], R2;
    double zw;
    double n[3], d;
    double h0, amp, wavelength;
} orc_geom;

/* ------------------------------------------------------------------------ */
/* lattice                                                                   */

static int opp_q(int q) {
    for (int p = 0; p < NQ; ++p)
        if (CXQ[p] == -CXQ[q] && CYQ[p] == -CYQ[q] && CZQ[p] == -CZQ[q]) return p;
    return -1;
}

static double w_q(int q) {
    int c2 = CXQ[q] * CXQ[q] + CYQ[q] * CYQ[q] + CZQ[q] * CZQ[q];
    return c2 == 0 ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
}

void orc_lattice(int *cx, int *cy, int *cz, double *w, int *opp) {
    for (int q = 0; q < NQ; ++q) {
        cx[q] = CXQ[q];
        cy[q] = CYQ[q];
        cz[q] = CZQ[q];
        w[q] = w_q(q);
        opp[q] = opp_q(q);
    }
}

static long cell(const orc_params *P, int x, int y, int z) {
    x %= P->nx; if (x < 0) x += P->nx;
    y %= P->ny; if (y < 0) y += P->ny;
    z %= P->nz; if (z < 0) z += P->nz;
    return (long)x + (long)P->nx * ((long)y + (long)P->ny * (long)z);
}

static void coords(const orc_params *P, long i, int *x, int *y, int *z) {
    *x = (int)(i % P->nx);
    *y = (int)((i / P->nx) % P->ny);
    *z = (int)(i / ((long)P->nx * P->ny));
}

static long ncell(const orc_params *P) { return (long)P->nx * P->ny * P->nz; }

static long nbr(const orc_params *P, long i, int dx, int dy, int dz) {
    int x, y, z;
    coords(P, i, &x, &y, &z);
    return cell(P, x + dx, y + dy, z + dz);
}

/* equilibrium (second-order D3Q19 form; the paper cites but does not print it) */
static double feq(int q, double rho, const double u[3]) {
    double cu = CXQ[q] * u[0] + CYQ[q] * u[1] + CZQ[q] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w_q(q) * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

/* moments rho = sum f, rho u = sum c f (Sec. II) */
static void moments(const double f[NQ], double *rho, double u[3]) {
    double r = 0, jx = 0, jy = 0, jz = 0;
    for (int q = 0; q < NQ; ++q) {
        r += f[q];
        jx += CXQ[q] * f[q];
        jy += CYQ[q] * f[q];
        jz += CZQ[q] * f[q];
    }
    *rho = r;
    u[0] = jx / r;
    u[1] = jy / r;
    u[2] = jz / r;
}

/* TRT collision (Sec. II, Eq. lbe2): even and odd parts relax with tau_e = tau
 * and tau_o = 1/2 + Lambda/(tau - 1/2); BGK is tau_o = tau_e. */
static void collide(const orc_params *P, const double f[NQ], double out[NQ]) {
    double rho, u[3];
    moments(f, &rho, u);
    double te = P->tau;
    double to = P->collision == 1 ? 0.5 + P->magic / (P->tau - 0.5) : P->tau;
    for (int q = 0; q < NQ; ++q) {
        int qb = opp_q(q);
        double fp = 0.5 * (f[q] + f[qb]), fm = 0.5 * (f[q] - f[qb]);
        double ep = 0.5 * (feq(q, rho, u) + feq(qb, rho, u));
        double em = 0.5 * (feq(q, rho, u) - feq(qb, rho, u));
        out[q] = f[q] - (fp - ep) / te - (fm - em) / to;
    }
}

void orc_collide(const orc_params *P, const double *f, double *out) { collide(P, f, out); }
double orc_feq(int q, double rho, const double *u) { return feq(q, rho, u); }

/* ------------------------------------------------------------------------ */
/* PLIC (Sec. II.B)                                                          */

/* Area of {(s,t) in [-1/2,1/2]^2 : al*s + be*t >= ga}: clip the square against
 * one half-plane (Sutherland-Hodgman) and apply the shoelace formula. */
static double clipped_square_area(double al, double be, double ga) {
    const double vx[4] = {-0.5, 0.5, 0.5, -0.5}, vy[4] = {-0.5, -0.5, 0.5, 0.5};
    double ox[8], oy[8];
    int n = 0;
    for (int i = 0; i < 4; ++i) {
        int j = (i + 1) % 4;
        double di = al * vx[i] + be * vy[i] - ga;
        double dj = al * vx[j] + be * vy[j] - ga;
        if (di >= 0) {
            ox[n] = vx[i];
            oy[n] = vy[i];
            ++n;
        }
        if ((di >= 0) != (dj >= 0)) {
            double s = di / (di - dj);
            ox[n] = vx[i] + s * (vx[j] - vx[i]);
            oy[n] = vy[i] + s * (vy[j] - vy[i]);
            ++n;
        }
    }
    double a2 = 0;
    for (int i = 0; i < n; ++i) {
        int j = (i + 1) % n;
        a2 += ox[i] * oy[j] - ox[j] * oy[i];
    }
    return 0.5 * a2;
}

/* vol(V cap P) for the unit cell V = [-1/2,1/2]^3 and the half-space
 * P = {y : (y - a n).n >= 0}, n a unit vector (Sec. II.B).
 * Divergence theorem with F(y) = y - a n, which vanishes in the normal
 * direction on the cut plane: 3 vol = sum over the six faces of
 * (F . outward normal) * (area of the face part inside P).
 * Pinned: brute-force sub-sampling, axis-aligned closed forms. */
double orc_plic_volume(const double *n, double a) {
    double vol = 0;
    for (int k = 0; k < 3; ++k) {
        int i = (k + 1) % 3, j = (k + 2) % 3;
        for (int side = -1; side <= 1; side += 2) {
            double area = clipped_square_area(n[i], n[j], a - n[k] * side * 0.5);
            vol += (0.5 - side * a * n[k]) * area;
        }
    }
    return vol / 3.0;
}

/* The offset a with vol(V cap P(a)) = phi, by bisection (Sec. II.B: the paper
 * takes 40 iterations; the oracle takes `iters`).  The volume falls from 1 at
 * a = -h to 0 at a = +h, h = (|n1|+|n2|+|n3|)/2.  phi is clamped to [0,1].
 * Pinned: round trip against orc_plic_volume, brute force. */
double orc_plic_offset(const double *n, double phi, int iters) {
    double h = 0.5 * (fabs(n[0]) + fabs(n[1]) + fabs(n[2]));
    if (phi <= 0) return h;
    if (phi >= 1) return -h;
    double lo = -h, hi = h;
    for (int it = 0; it < iters; ++it) {
        double mid = 0.5 * (lo + hi);
        if (orc_plic_volume(n, mid) > phi) lo = mid;
        else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* ------------------------------------------------------------------------ */
/* fill level at obstacle cells (Sec. II.A, reflection with aperture alpha)  */

/* phi(x_o) = sum |n_w.c_q| phi(x_o+c_q) / sum |n_w.c_q| over the D3Q19
 * neighbours that are not obstacle and pass |n_w.c_q/|c_q|| > sqrt(2)/2.
 * Readings: n_w is the sum of the lattice vectors to the non-obstacle
 * neighbours (integer); the aperture test is done exactly in integers,
 * 2 (N.c)^2 > |N|^2 |c|^2; gas cells count with phi = 0; 0/0 gives 0. */
static double reflect_phi(const orc_params *P, const uint8_t *flags, const double *phi, long o) {
    int N[3] = {0, 0, 0};
    for (int q = 1; q < NQ; ++q) {
        long y = nbr(P, o, CXQ[q], CYQ[q], CZQ[q]);
        if (flags[y] & FL_OBS) continue;
        N[0] += CXQ[q];
        N[1] += CYQ[q];
        N[2] += CZQ[q];
    }
    long N2 = (long)N[0] * N[0] + (long)N[1] * N[1] + (long)N[2] * N[2];
    if (N2 == 0) return 0.0;
    double num = 0, den = 0;
    for (int q = 1; q < NQ; ++q) {
        long y = nbr(P, o, CXQ[q], CYQ[q], CZQ[q]);
        if (flags[y] & FL_OBS) continue;
        long dot = (long)N[0] * CXQ[q] + (long)N[1] * CYQ[q] + (long)N[2] * CZQ[q];
        long c2 = CXQ[q] * CXQ[q] + CYQ[q] * CYQ[q] + CZQ[q] * CZQ[q];
        if (2 * dot * dot > N2 * c2) {
            double wgt = fabs((double)dot) / sqrt((double)(N2 * c2));
            num += wgt * phi[y];
            den += wgt;
        }
    }
    return den > 0 ? num / den : 0.0;
}

/* phi with obstacle cells replaced by their reflected value */
static void extend_phi(const orc_params *P, const uint8_t *flags, const double *phi, double *ext) {
    long N = ncell(P);
    for (long i = 0; i < N; ++i) ext[i] = (flags[i] & FL_OBS) ? reflect_phi(P, flags, phi, i) : phi[i];
}

void orc_reflect_phi(const orc_params *P, const uint8_t *flags, const double *phi, double *ext) {
    extend_phi(P, flags, phi, ext);
}

/* Parker-Youngs gradient (Sec. II.A, Eq. normal): central difference across
 * the cell, smoothed transversally with weights 4 (face), 2 (edge), 1 (corner). */
static void parker_youngs(const orc_params *P, const double *g, long i, double n[3]) {
    n[0] = n[1] = n[2] = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                double v = g[nbr(P, i, dx, dy, dz)];
                if (dx != 0) n[0] += dx * (dy == 0 ? 2 : 1) * (dz == 0 ? 2 : 1) * v;
                if (dy != 0) n[1] += dy * (dx == 0 ? 2 : 1) * (dz == 0 ? 2 : 1) * v;
                if (dz != 0) n[2] += dz * (dx == 0 ? 2 : 1) * (dy == 0 ? 2 : 1) * v;
            }
}

static int unit(double v[3]) {
    double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (l < 1e-12) {
        v[0] = v[1] = v[2] = 0;
        return 0;
    }
    v[0] /= l;
    v[1] /= l;
    v[2] /= l;
    return 1;
}

static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* unit wall normal at a fluid cell, pointing into the wall: the normalised sum
 * of the lattice vectors to its obstacle neighbours (reading). 0 if none. */
static int wall_normal(const orc_params *P, const uint8_t *flags, long i, double nw[3]) {
    nw[0] = nw[1] = nw[2] = 0;
    int cnt = 0;
    for (int q = 1; q < NQ; ++q) {
        long y = nbr(P, i, CXQ[q], CYQ[q], CZQ[q]);
        if (flags[y] & FL_OBS) {
            nw[0] += CXQ[q];
            nw[1] += CYQ[q];
            nw[2] += CZQ[q];
            ++cnt;
        }
    }
    if (!cnt) return 0;
    return unit(nw);
}

/* Interface normals and PLIC offsets (Sec. II.B): for every interface cell,
 * n = Parker-Youngs(phi with reflected obstacle values), nh = n/|n|, and the
 * offset a with vol(V cap P) = phi.  Output normal4[4i..4i+3] = (nh, a);
 * cells that are not interface, or with |n| < 1e-12, get (0,0,0,0).
 * Pinned: plane and sphere fields (via the curvature pins). */
void orc_normals(const orc_params *P, const uint8_t *flags, const double *phi, double *normal4, int iters) {
    long N = ncell(P);
    double *ext = (double *)malloc(sizeof(double) * N);
    extend_phi(P, flags, phi, ext);
    for (long i = 0; i < N; ++i) {
        normal4[4 * i] = normal4[4 * i + 1] = normal4[4 * i + 2] = normal4[4 * i + 3] = 0;
        if (!(flags[i] & FL_IF)) continue;
        double n[3];
        parker_youngs(P, ext, i, n);
        if (!unit(n)) continue;
        normal4[4 * i] = n[0];
        normal4[4 * i + 1] = n[1];
        normal4[4 * i + 2] = n[2];
        normal4[4 * i + 3] = orc_plic_offset(n, phi[i], iters);
    }
    free(ext);
}

/* ------------------------------------------------------------------------ */
/* dense linear least squares (Householder QR), with equality constraints    */

/* Solve min |A x - b| (m x k, row-major, m >= k) by Householder QR.  Returns 0
 * and x on success; 1 if some |R_jj| <= rtol * max|R_ii| (rank deficient). */
static int householder_ls(int m, int k, double *A, double *b, double *x, double rtol) {
    for (int j = 0; j < k; ++j) {
        double nrm = 0;
        for (int i = j; i < m; ++i) nrm += A[i * k + j] * A[i * k + j];
        nrm = sqrt(nrm);
        if (nrm == 0) continue;
        double alpha = A[j * k + j] > 0 ? -nrm : nrm;
        /* v = a_j - alpha e_j, stored in place below the diagonal */
        double v0 = A[j * k + j] - alpha;
        double vnorm2 = v0 * v0;
        for (int i = j + 1; i < m; ++i) vnorm2 += A[i * k + j] * A[i * k + j];
        if (vnorm2 == 0) continue;
        for (int c = j + 1; c < k; ++c) {
            double s = v0 * A[j * k + c];
            for (int i = j + 1; i < m; ++i) s += A[i * k + j] * A[i * k + c];
            s = 2 * s / vnorm2;
            A[j * k + c] -= s * v0;
            for (int i = j + 1; i < m; ++i) A[i * k + c] -= s * A[i * k + j];
        }
        double s = v0 * b[j];
        for (int i = j + 1; i < m; ++i) s += A[i * k + j] * b[i];
        s = 2 * s / vnorm2;
        b[j] -= s * v0;
        for (int i = j + 1; i < m; ++i) b[i] -= s * A[i * k + j];
        A[j * k + j] = alpha;
        for (int i = j + 1; i < m; ++i) A[i * k + j] = 0;
    }
    double rmax = 0;
    for (int j = 0; j < k; ++j) rmax = fmax(rmax, fabs(A[j * k + j]));
    if (rmax == 0) return 1;
    for (int j = 0; j < k; ++j)
        if (fabs(A[j * k + j]) <= rtol * rmax) return 1;
    for (int j = k - 1; j >= 0; --j) {
        double s = b[j];
        for (int c = j + 1; c < k; ++c) s -= A[j * k + c] * x[c];
        x[j] = s / A[j * k + j];
    }
    return 0;
}

/* min |A x - b| subject to C x = d (nc <= 2 rows, full row rank) by the
 * null-space method: C^T = Q R (Householder, explicit Q), x = Q1 R^-T d + Q2 z,
 * then an unconstrained fit for z.  Returns 0 on success, 1 if the reduced
 * least-squares problem is rank deficient or has fewer rows than unknowns. */
static int constrained_ls(int m, int k, const double *A, const double *b, int nc, const double *C,
                          const double *d, double *x, double rtol) {
    double Q[36], R[4] = {0, 0, 0, 0};
    /* Q = I (k x k) */
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Q[i * k + j] = (i == j);
    double Ct[12]; /* k x nc */
    for (int i = 0; i < k; ++i)
        for (int r = 0; r < nc; ++r) Ct[i * nc + r] = C[r * k + i];
    for (int j = 0; j < nc; ++j) {
        double nrm = 0;
        for (int i = j; i < k; ++i) nrm += Ct[i * nc + j] * Ct[i * nc + j];
        nrm = sqrt(nrm);
        if (nrm == 0) return 1;
        double alpha = Ct[j * nc + j] > 0 ? -nrm : nrm;
        double v[6] = {0, 0, 0, 0, 0, 0};
        v[j] = Ct[j * nc + j] - alpha;
        for (int i = j + 1; i < k; ++i) v[i] = Ct[i * nc + j];
        double vn2 = 0;
        for (int i = j; i < k; ++i) vn2 += v[i] * v[i];
        if (vn2 == 0) continue;
        for (int c = 0; c < nc; ++c) { /* H Ct */
            double s = 0;
            for (int i = j; i < k; ++i) s += v[i] * Ct[i * nc + c];
            s = 2 * s / vn2;
            for (int i = j; i < k; ++i) Ct[i * nc + c] -= s * v[i];
        }
        for (int r = 0; r < k; ++r) { /* Q = Q H */
            double s = 0;
            for (int i = j; i < k; ++i) s += Q[r * k + i] * v[i];
            s = 2 * s / vn2;
            for (int i = j; i < k; ++i) Q[r * k + i] -= s * v[i];
        }
    }
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nc; ++j) R[i * nc + j] = Ct[i * nc + j];
    /* R^T y1 = d (forward substitution) */
    double y1[2];
    for (int i = 0; i < nc; ++i) {
        double s = d[i];
        for (int j = 0; j < i; ++j) s -= R[j * nc + i] * y1[j];
        if (R[i * nc + i] == 0) return 1;
        y1[i] = s / R[i * nc + i];
    }
    double x0[6] = {0, 0, 0, 0, 0, 0};
    for (int r = 0; r < k; ++r)
        for (int i = 0; i < nc; ++i) x0[r] += Q[r * k + i] * y1[i];
    int kr = k - nc;
    if (m < kr) return 1;
    if (kr == 0) {
        for (int r = 0; r < k; ++r) x[r] = x0[r];
        return 0;
    }
    double *Ar = (double *)malloc(sizeof(double) * (m > 0 ? m : 1) * kr);
    double *br = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    for (int i = 0; i < m; ++i) {
        double ax0 = 0;
        for (int c = 0; c < k; ++c) ax0 += A[i * k + c] * x0[c];
        br[i] = b[i] - ax0;
        for (int j = 0; j < kr; ++j) {
            double s = 0;
            for (int c = 0; c < k; ++c) s += A[i * k + c] * Q[c * k + nc + j];
            Ar[i * kr + j] = s;
        }
    }
    double z[6];
    int bad = householder_ls(m, kr, Ar, br, z, rtol);
    free(Ar);
    free(br);
    if (bad) return 1;
    for (int r = 0; r < k; ++r) {
        x[r] = x0[r];
        for (int j = 0; j < kr; ++j) x[r] += Q[r * k + nc + j] * z[j];
    }
    return 0;
}

#define LS_RTOL 1e-6

/* Fit of the model f(u,v) = A u^2 + B v^2 + C uv + H u + I v (J = 0,
 * Sec. II.C Eqs. LSQR-model, LSQR-error) to m rows (u^2, v^2, uv, u, v) -> f,
 * with nc (0 or 2) equality rows from the contact constraint at the centre
 * cell (Eq. contactConstraint).  Fallback chain (reading): full model; if it
 * has too few rows or is rank deficient, the isotropic model B = A, C = 0;
 * if that fails too, all coefficients 0.  mode_out = 0 full, 1 reduced, 2 zero.
 * coef = (A, B, C, H, I).  Pinned: exact paraboloid point sets. */
int orc_ls_fit(int m, const double *rows, const double *rhs, int nc, const double *crow, const double *crhs,
               double *coef, int *mode_out) {
    for (int i = 0; i < 5; ++i) coef[i] = 0;
    int ok = 0;
    if (m >= 5 - nc && m > 0) {
        double *A = (double *)malloc(sizeof(double) * m * 5);
        double *b = (double *)malloc(sizeof(double) * m);
        memcpy(A, rows, sizeof(double) * m * 5);
        memcpy(b, rhs, sizeof(double) * m);
        if (nc == 0) ok = !householder_ls(m, 5, A, b, coef, LS_RTOL);
        else ok = !constrained_ls(m, 5, A, b, nc, crow, crhs, coef, LS_RTOL);
        free(A);
        free(b);
        if (ok) {
            if (mode_out) *mode_out = 0;
            return 0;
        }
    }
    /* isotropic model: unknowns (A, H, I); full = M red with A=B, C=0 */
    if (m >= 3 - nc && m > 0) {
        double *A = (double *)malloc(sizeof(double) * m * 3);
        double *b = (double *)malloc(sizeof(double) * m);
        for (int i = 0; i < m; ++i) {
            const double *r = rows + 5 * i;
            A[3 * i] = r[0] + r[1];
            A[3 * i + 1] = r[3];
            A[3 * i + 2] = r[4];
            b[i] = rhs[i];
        }
        double Cr[6], x3[3] = {0, 0, 0};
        for (int i = 0; i < nc; ++i) {
            const double *r = crow + 5 * i;
            Cr[3 * i] = r[0] + r[1];
            Cr[3 * i + 1] = r[3];
            Cr[3 * i + 2] = r[4];
        }
        if (nc == 0) ok = !householder_ls(m, 3, A, b, x3, LS_RTOL);
        else ok = !constrained_ls(m, 3, A, b, nc, Cr, crhs, x3, LS_RTOL);
        free(A);
        free(b);
        if (ok) {
            coef[0] = x3[0];
            coef[1] = x3[0];
            coef[2] = 0;
            coef[3] = x3[1];
            coef[4] = x3[2];
            if (mode_out) *mode_out = 1;
            return 1;
        }
    }
    if (mode_out) *mode_out = 2;
    return 2;
}

/* Mean curvature of the graph of f at (0,0), Eq. (anacurv) with the mixed term
 * -C H I (reading: the printed -2CHI does not match the differential-geometry
 * mean curvature of f with the C uv term; the two agree when H I = 0).
 * Pinned: closed-form mean curvature of tilted quadrics. */
double orc_kappa_from_coef(const double *c) {
    double A = c[0], B = c[1], C = c[2], H = c[3], I = c[4];
    double g = 1 + H * H + I * I;
    return (A * (1 + I * I) + B * (1 + H * H) - C * H * I) / (g * sqrt(g));
}

/* contact point and contact normal of contact-line cell j (Sec. II.C, Fig.
 * contactPoint, Eq. contactNormal).  o: offset of j from the centre cell;
 * nj, aj: its PLIC normal and offset; nw: its unit wall normal (into the wall).
 * Readings: the wall plane is half way to the obstacle neighbour,
 * (y - o).nw = 1/2; the contact point is p_j moved inside the PLIC plane along
 * the projection d of nw onto that plane; no contact point if |d| < 1e-6.
 * m = nw cos(theta) + nt sin(theta), nt = unit projection of nj onto the wall. */
static int contact_point(const double o[3], const double nj[3], double aj, const double nw[3], double theta,
                         double pc[3], double mh[3]) {
    double pj[3] = {o[0] + aj * nj[0], o[1] + aj * nj[1], o[2] + aj * nj[2]};
    double wn = dot3(nw, nj);
    double d[3] = {nw[0] - wn * nj[0], nw[1] - wn * nj[1], nw[2] - wn * nj[2]};
    double dl = sqrt(dot3(d, d));
    if (dl < 1e-6) return 0;
    for (int k = 0; k < 3; ++k) d[k] /= dl;
    double rel[3] = {pj[0] - o[0], pj[1] - o[1], pj[2] - o[2]};
    double s = (0.5 - dot3(rel, nw)) / dot3(d, nw);
    for (int k = 0; k < 3; ++k) pc[k] = pj[k] + s * d[k];
    double nt[3] = {nj[0] - wn * nw[0], nj[1] - wn * nw[1], nj[2] - wn * nw[2]};
    if (!unit(nt)) return 0;
    for (int k = 0; k < 3; ++k) mh[k] = nw[k] * cos(theta) + nt[k] * sin(theta);
    return 1;
}

/* LSQR curvature of interface cell i (Sec. II.C).  normal4 from orc_normals.
 * info[0] = rows, info[1] = fit mode, info[2] = 1 if centre constraint. */
static double lsqr_cell(const orc_params *P, const uint8_t *flags, const double *normal4, long i, int info[3]) {
    const double *ni = normal4 + 4 * i;
    double n[3] = {ni[0], ni[1], ni[2]}, a = ni[3];
    info[0] = info[1] = info[2] = 0;
    if (n[0] == 0 && n[1] == 0 && n[2] == 0) {
        info[1] = 2;
        return 0;
    }
    /* local frame: t_u from the axis with the smallest |n_k| (lowest index on ties) */
    int k = 0;
    for (int j = 1; j < 3; ++j)
        if (fabs(n[j]) < fabs(n[k])) k = j;
    double e[3] = {0, 0, 0};
    e[k] = 1;
    double tu[3], tv[3];
    cross3(e, n, tu);
    unit(tu);
    cross3(n, tu, tv);
    double p[3] = {a * n[0], a * n[1], a * n[2]};

    double rows[5 * 80], rhs[80], crow[10], crhs[2];
    int m = 0, nc = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                long j = nbr(P, i, dx, dy, dz);
                if (!(flags[j] & FL_IF)) continue;
                const double *nj4 = normal4 + 4 * j;
                double nj[3] = {nj4[0], nj4[1], nj4[2]};
                if (nj[0] == 0 && nj[1] == 0 && nj[2] == 0) continue;
                double o[3] = {dx, dy, dz};
                int centre = (dx == 0 && dy == 0 && dz == 0);
                if (!centre) {
                    double dv[3] = {o[0] + nj4[3] * nj[0] - p[0], o[1] + nj4[3] * nj[1] - p[1],
                                    o[2] + nj4[3] * nj[2] - p[2]};
                    double u = dot3(dv, tu), v = dot3(dv, tv), f = dot3(dv, n);
                    double *r = rows + 5 * m;
                    r[0] = u * u;
                    r[1] = v * v;
                    r[2] = u * v;
                    r[3] = u;
                    r[4] = v;
                    rhs[m++] = f;
                }
                double nw[3];
                if (!wall_normal(P, flags, j, nw)) continue;
                double pc[3], mh[3];
                if (!contact_point(o, nj, nj4[3], nw, P->theta, pc, mh)) continue;
                double mn = dot3(mh, n);
                if (fabs(mn) < 1e-6) continue;
                double dc[3] = {pc[0] - p[0], pc[1] - p[1], pc[2] - p[2]};
                double uc = dot3(dc, tu), vc = dot3(dc, tv);
                double gu = -dot3(mh, tu) / mn, gv = -dot3(mh, tv) / mn;
                /* grad f(uc,vc) = (2A uc + C vc + H, 2B vc + C uc + I) */
                double r1[5] = {2 * uc, 0, vc, 1, 0}, r2[5] = {0, 2 * vc, uc, 0, 1};
                if (centre) {
                    memcpy(crow, r1, sizeof r1);
                    memcpy(crow + 5, r2, sizeof r2);
                    crhs[0] = gu;
                    crhs[1] = gv;
                    nc = 2;
                } else {
                    memcpy(rows + 5 * m, r1, sizeof r1);
                    rhs[m++] = gu;
                    memcpy(rows + 5 * m, r2, sizeof r2);
                    rhs[m++] = gv;
                }
            }
    double coef[5];
    int mode;
    orc_ls_fit(m, rows, rhs, nc, crow, crhs, coef, &mode);
    info[0] = m;
    info[1] = mode;
    info[2] = nc > 0;
    return orc_kappa_from_coef(coef);
}

/* ------------------------------------------------------------------------ */
/* TR curvature (Sec. II.B, triangle fan of PLIC points after Pohl, curvature */
/* after Taubin)                                                             */

/* Mean curvature at the origin of a fan of m points given in the tangent
 * frame of the centre point (u, v along the tangent plane, h along the
 * centre normal, which points towards the liquid).  Readings of the two cited
 * steps, which the paper does not spell out:
 *  - fan: the points ordered by their angle atan2(v, u) around the normal
 *    (ties by the index key[]), consecutive points joined with the centre
 *    into triangles, cyclically; a pair whose angular gap is >= pi is not
 *    joined (the fan is open there); points whose projection lies within
 *    1e-6 of the centre are dropped;
 *  - curvature: the normal curvature along each edge, kappa_j = 2 h_j /
 *    |p_j|^2 (the circle through the centre, tangent to its plane, that
 *    passes through p_j), averaged with weights equal to the summed areas of
 *    the fan triangles that hold edge j (Taubin's weights; the trace of his
 *    curvature tensor is this mean).
 * Returns 0 if no triangle is formed.  Pinned: exact sphere and plane point
 * sets, symmetric rings on quadrics (mean curvature A + B), uneven rings. */
double orc_tr_fan(int m, const double *u, const double *v, const double *h, const int *key) {
    double ang[27], kap[27], pu[27], pv[27], ph[27];
    int kk[27], n = 0;
    for (int j = 0; j < m && n < 27; ++j) {
        double r2 = u[j] * u[j] + v[j] * v[j];
        if (r2 < 1e-12) continue;
        /* insertion by (angle, key) */
        double a = atan2(v[j], u[j]);
        int pos = n;
        while (pos > 0 && (ang[pos - 1] > a || (ang[pos - 1] == a && kk[pos - 1] > key[j]))) {
            ang[pos] = ang[pos - 1];
            kap[pos] = kap[pos - 1];
            pu[pos] = pu[pos - 1];
            pv[pos] = pv[pos - 1];
            ph[pos] = ph[pos - 1];
            kk[pos] = kk[pos - 1];
            --pos;
        }
        ang[pos] = a;
        kap[pos] = 2.0 * h[j] / (r2 + h[j] * h[j]);
        pu[pos] = u[j];
        pv[pos] = v[j];
        ph[pos] = h[j];
        kk[pos] = key[j];
        ++n;
    }
    if (n < 2) return 0.0;
    const double pi = 3.14159265358979323846;
    double num = 0, den = 0;
    for (int k = 0; k < n; ++k) {
        int s = (k + 1) % n;
        double gap = ang[s] - ang[k];
        if (s == 0) gap += 2.0 * pi;
        if (gap >= pi) continue;
        double a[3] = {pu[k], pv[k], ph[k]}, b[3] = {pu[s], pv[s], ph[s]}, c[3];
        cross3(a, b, c);
        double area = 0.5 * sqrt(dot3(c, c));
        num += area * (kap[k] + kap[s]);
        den += 2.0 * area;
    }
    return den > 0 ? num / den : 0.0;
}

/* TR curvature of interface cell i: the PLIC points p_j = x_j + a_j n_j of
 * the other interface cells of the 3x3x3 block (nonzero normal; the same
 * points as the LSQR fit, reading O20/O21) relative to the centre point,
 * in the centre's frame (the LSQR frame rule), through orc_tr_fan with the
 * block position (dz+1)*9 + (dy+1)*3 + (dx+1) as the tie key.  No wetting
 * treatment (the paper leaves TR without one).  normal4 from orc_normals.
 * Pinned: see orc_tr_fan; sub-sampled spheres; cube symmetry. */
double orc_tr_cell(const orc_params *P, const uint8_t *flags, const double *normal4, long i) {
    const double *ni = normal4 + 4 * i;
    double n[3] = {ni[0], ni[1], ni[2]}, a = ni[3];
    if (n[0] == 0 && n[1] == 0 && n[2] == 0) return 0.0;
    int k = 0;
    for (int j = 1; j < 3; ++j)
        if (fabs(n[j]) < fabs(n[k])) k = j;
    double e[3] = {0, 0, 0};
    e[k] = 1;
    double tu[3], tv[3];
    cross3(e, n, tu);
    unit(tu);
    cross3(n, tu, tv);
    double p[3] = {a * n[0], a * n[1], a * n[2]};
    double u[27], v[27], h[27];
    int key[27], m = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (dx == 0 && dy == 0 && dz == 0) continue;
                long j = nbr(P, i, dx, dy, dz);
                if (!(flags[j] & FL_IF)) continue;
                const double *nj = normal4 + 4 * j;
                if (nj[0] == 0 && nj[1] == 0 && nj[2] == 0) continue;
                double d[3] = {dx + nj[3] * nj[0] - p[0], dy + nj[3] * nj[1] - p[1], dz + nj[3] * nj[2] - p[2]};
                u[m] = dot3(d, tu);
                v[m] = dot3(d, tv);
                h[m] = dot3(d, n);
                key[m] = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                ++m;
            }
    return orc_tr_fan(m, u, v, h, key);
}

/* ------------------------------------------------------------------------ */
/* FD curvature (Sec. II.A)                                                 */

/* K8 kernel (1 - r^2/eps^2)^4 with eps = 2 on the 3x3x3 stencil, normalised
 * by its discrete sum (reading of "support radius 2: only next neighbours"). */
static double k8(int dx, int dy, int dz) {
    double r2 = dx * dx + dy * dy + dz * dz;
    double t = 1.0 - r2 / 4.0;
    return t * t * t * t;
}

/* FD curvature field kappa = -1/2 div(nh) (Eq. curvature; the factor 1/2 is a
 * reading so that a sphere gives its mean curvature 1/R, as p_s = 2 sigma
 * kappa requires).  Steps: (1) phi with reflected obstacle values; (2) K8
 * smoothing at non-obstacle cells, reflection of the smoothed field at
 * obstacle cells; (3) Parker-Youngs normals nh of the smoothed field at
 * non-obstacle cells; at obstacle cells the wetting normal of Eq.
 * contactNormal, nw cos(theta) + nt sin(theta), nw into the wall, nt the unit
 * projection onto the wall of nh at the neighbour x_b most aligned with the
 * outward wall normal; (4) central differences of nh.  kappa is written for
 * interface cells only.  Pinned: linear fields, smooth spheres, symmetry. */
static void fd_curvature(const orc_params *P, const uint8_t *flags, const double *phi, double *kappa) {
    long N = ncell(P);
    double *ext = (double *)malloc(sizeof(double) * N);
    double *sm = (double *)malloc(sizeof(double) * N);
    double *nh = (double *)malloc(sizeof(double) * 3 * N);
    extend_phi(P, flags, phi, ext);
    double wsum = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) wsum += k8(dx, dy, dz);
    for (long i = 0; i < N; ++i) {
        sm[i] = 0;
        if (flags[i] & FL_OBS) continue;
        double s = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) s += k8(dx, dy, dz) * ext[nbr(P, i, dx, dy, dz)];
        sm[i] = s / wsum;
    }
    for (long i = 0; i < N; ++i)
        if (flags[i] & FL_OBS) sm[i] = reflect_phi(P, flags, sm, i);
    for (long i = 0; i < N; ++i) {
        nh[3 * i] = nh[3 * i + 1] = nh[3 * i + 2] = 0;
        if (flags[i] & FL_OBS) continue;
        double n[3];
        parker_youngs(P, sm, i, n);
        unit(n);
        nh[3 * i] = n[0];
        nh[3 * i + 1] = n[1];
        nh[3 * i + 2] = n[2];
    }
    for (long o = 0; o < N; ++o) {
        if (!(flags[o] & FL_OBS)) continue;
        int Nv[3] = {0, 0, 0}, best = -1;
        double bestv = -1e300;
        for (int q = 1; q < NQ; ++q) {
            long y = nbr(P, o, CXQ[q], CYQ[q], CZQ[q]);
            if (flags[y] & FL_OBS) continue;
            Nv[0] += CXQ[q];
            Nv[1] += CYQ[q];
            Nv[2] += CZQ[q];
        }
        if (Nv[0] == 0 && Nv[1] == 0 && Nv[2] == 0) continue;
        for (int q = 1; q < NQ; ++q) {
            long y = nbr(P, o, CXQ[q], CYQ[q], CZQ[q]);
            if (flags[y] & FL_OBS) continue;
            double c2 = CXQ[q] * CXQ[q] + CYQ[q] * CYQ[q] + CZQ[q] * CZQ[q];
            double v = (Nv[0] * CXQ[q] + Nv[1] * CYQ[q] + Nv[2] * CZQ[q]) / sqrt(c2);
            if (v > bestv) {
                bestv = v;
                best = q;
            }
        }
        double nw[3] = {-(double)Nv[0], -(double)Nv[1], -(double)Nv[2]};
        unit(nw);
        long xb = nbr(P, o, CXQ[best], CYQ[best], CZQ[best]);
        double nb[3] = {nh[3 * xb], nh[3 * xb + 1], nh[3 * xb + 2]};
        double wn = dot3(nb, nw);
        double nt[3] = {nb[0] - wn * nw[0], nb[1] - wn * nw[1], nb[2] - wn * nw[2]};
        unit(nt);
        for (int k = 0; k < 3; ++k) nh[3 * o + k] = nw[k] * cos(P->theta) + nt[k] * sin(P->theta);
    }
    for (long i = 0; i < N; ++i) {
        if (!(flags[i] & FL_IF)) {
            kappa[i] = 0;
            continue;
        }
        double div = 0;
        div += nh[3 * nbr(P, i, 1, 0, 0)] - nh[3 * nbr(P, i, -1, 0, 0)];
        div += nh[3 * nbr(P, i, 0, 1, 0) + 1] - nh[3 * nbr(P, i, 0, -1, 0) + 1];
        div += nh[3 * nbr(P, i, 0, 0, 1) + 2] - nh[3 * nbr(P, i, 0, 0, -1) + 2];
        kappa[i] = -0.5 * (div / 2.0);
    }
    free(ext);
    free(sm);
    free(nh);
}

/* Curvature of every interface cell from phi (model P->curv_model); writes
 * kappa[N] (0 outside interface cells) and normal4[4N] (always the PLIC
 * normals, which the corner rule of the step uses).  stats[0..2] = cells
 * fitted with the full / isotropic / zero model, stats[3] = centre-constrained
 * cells (LSQR only).  Pinned: see the LSQR and FD functions above. */
void orc_curvature(const orc_params *P, const uint8_t *flags, const double *phi, double *kappa, double *normal4,
                   int plic_iters, long *stats) {
    long N = ncell(P);
    for (int s = 0; s < 4; ++s) stats[s] = 0;
    orc_normals(P, flags, phi, normal4, plic_iters);
    if (P->curv_model == 1) {
        fd_curvature(P, flags, phi, kappa);
        return;
    }
    if (P->curv_model == 4) {
        for (long i = 0; i < N; ++i) kappa[i] = (flags[i] & FL_IF) ? orc_tr_cell(P, flags, normal4, i) : 0.0;
        return;
    }
    for (long i = 0; i < N; ++i) {
        kappa[i] = 0;
        if (!(flags[i] & FL_IF) || P->curv_model == 2) continue;
        int info[3];
        kappa[i] = lsqr_cell(P, flags, normal4, i, info);
        stats[info[1]]++;
        stats[3] += info[2];
    }
}

/* ------------------------------------------------------------------------ */
/* the time step                                                            */

/* One FSLBM step t -> t+1 after the curvature kappa(t) is known.
 *   fin      post-collision PDFs f'(t), 19*N
 *   fout     post-collision PDFs f'(t+1) (fluid cells written)
 *   flags    cell types at t; overwritten with the types at t+1
 *   mass     m(t) -> m(t+1) (interface entries meaningful)
 *   phi      phi(t) -> phi(t+1)
 *   kappa    kappa(t) (interface entries)
 *   normal4  PLIC normals at t (for the corner rule)
 *   rho      rho(t+1) of fluid cells (output)
 *   lost     mass that found no interface neighbour to go to (accumulated)
 *   counts   [liquid, interface, gas, filled, emptied, new interface from gas,
 *             interface from liquid, interface cells without liquid or
 *             without gas neighbour, liquid cells touching gas]
 * Steps: stream with the free-boundary condition Eq. (reconstruct) on gas
 * links and, at contact-line (corner) cells, on obstacle links whose outgoing
 * direction points against the interface normal projected into the wall
 * (Sec. II, Fig. inhomo); bounce-back on the other obstacle links; mass
 * exchange Eqs. (advection1, advection2); collision; conversion and excess
 * mass (cited by the paper from Koerner et al.; readings: conversion if
 * m > (1+eps) rho or m < -eps rho, filling beats emptying, new interface cells
 * from gas get f = feq(mean rho, mean u) of their fluid neighbours and m = 0,
 * liquid neighbours of emptied cells become interface with m = rho, excess
 * mass is shared equally by the interface neighbours after conversion).
 * With P->frozen the conversion test is skipped: no cell changes type, and
 * the step is a smooth function of (f', m, phi, sigma, theta) (the reading
 * of the adjoint windows; central differences of it give the FP64 reference
 * gradient).
 * Pinned: rest state, uniform flow, shear-wave decay, exact mass
 * conservation, invariants; the conversion readings on flat-interface
 * scenarios whose outcome follows from them by counting; the frozen step
 * equals the plain step where nothing converts. */
void orc_step(const orc_params *P, const double *fin, double *fout, uint8_t *flags, double *mass, double *phi,
              const double *kappa, const double *normal4, double *rho, double *lost, long *counts) {
    long N = ncell(P);
    uint8_t *ft = (uint8_t *)malloc(N);
    memcpy(ft, flags, N); /* types at time t */
    signed char *conv = (signed char *)calloc(N, 1);  /* 1 fill, 2 empty */
    signed char *newif = (signed char *)calloc(N, 1); /* 1 from gas, 2 from liquid */
    double *mnew = (double *)malloc(sizeof(double) * N);
    for (int c = 0; c < 9; ++c) counts[c] = 0;

    for (long x = 0; x < N; ++x) {
        mnew[x] = mass[x];
        if (!(ft[x] & (FL_LIQ | FL_IF))) continue;
        int is_if = (ft[x] & FL_IF) != 0;
        double fo[NQ], fs[NQ], rho0, u0[3];
        for (int q = 0; q < NQ; ++q) fo[q] = fin[(long)q * N + x];
        moments(fo, &rho0, u0); /* u_b: velocity of x at time t */
        double kap = is_if ? kappa[x] : 0.0;
        double rho_b = 3.0 * P->p_gas + 6.0 * P->sigma * kap; /* (p_g + 2 sigma kappa)/c_s^2 */
        int has_gas = 0, has_obs = 0;
        for (int q = 1; q < NQ; ++q) {
            uint8_t t = ft[nbr(P, x, CXQ[q], CYQ[q], CZQ[q])];
            has_gas |= (t & FL_GAS) != 0;
            has_obs |= (t & FL_OBS) != 0;
        }
        int corner = is_if && has_gas && has_obs;
        double ntan[3] = {0, 0, 0};
        if (corner) {
            double nw[3];
            wall_normal(P, ft, x, nw);
            const double *n4 = normal4 + 4 * x;
            double wn = n4[0] * nw[0] + n4[1] * nw[1] + n4[2] * nw[2];
            for (int k = 0; k < 3; ++k) ntan[k] = n4[k] - wn * nw[k];
        }
        double dm = 0;
        fs[0] = fo[0];
        for (int q = 1; q < NQ; ++q) {
            int qb = opp_q(q);
            long y = nbr(P, x, -CXQ[q], -CYQ[q], -CZQ[q]); /* source of direction q */
            uint8_t ty = ft[y];
            if (ty & (FL_LIQ | FL_IF)) {
                fs[q] = fin[(long)q * N + y];
                double k = (ty & FL_LIQ) ? 1.0 : 0.5 * (phi[x] + phi[y]);
                dm += k * (fin[(long)q * N + y] - fo[qb]);
            } else if (ty & FL_OBS) {
                double out = CXQ[qb] * ntan[0] + CYQ[qb] * ntan[1] + CZQ[qb] * ntan[2];
                if (corner && out < 0)
                    fs[q] = feq(q, rho_b, u0) + feq(qb, rho_b, u0) - fo[qb];
                else
                    fs[q] = fo[qb];
            } else {
                fs[q] = feq(q, rho_b, u0) + feq(qb, rho_b, u0) - fo[qb];
            }
        }
        double fc[NQ], r, u[3];
        moments(fs, &r, u);
        collide(P, fs, fc);
        for (int q = 0; q < NQ; ++q) fout[(long)q * N + x] = fc[q];
        rho[x] = r;
        if (is_if) {
            if (P->literal_phi) {
                double ph = phi[x] + dm / r;
                mnew[x] = ph * r;
            } else {
                mnew[x] = mass[x] + dm;
            }
            if (P->frozen) continue; /* types frozen: m and phi leave [0, rho] freely */
            if (mnew[x] > (1.0 + P->eps) * r) conv[x] = 1;
            else if (mnew[x] < -P->eps * r) conv[x] = 2;
        }
    }
    /* filling beats emptying */
    for (long x = 0; x < N; ++x) {
        if (conv[x] != 2) continue;
        for (int q = 1; q < NQ; ++q)
            if (conv[nbr(P, x, CXQ[q], CYQ[q], CZQ[q])] == 1) {
                conv[x] = 0;
                break;
            }
    }
    for (long x = 0; x < N; ++x) {
        if (!conv[x]) continue;
        for (int q = 1; q < NQ; ++q) {
            long y = nbr(P, x, CXQ[q], CYQ[q], CZQ[q]);
            if (conv[x] == 1 && (ft[y] & FL_GAS)) newif[y] = 1;
            if (conv[x] == 2 && (ft[y] & FL_LIQ)) newif[y] = 2;
        }
    }
    for (long y = 0; y < N; ++y) {
        if (newif[y] == 1) {
            double rs = 0, us[3] = {0, 0, 0};
            int cnt = 0;
            for (int q = 1; q < NQ; ++q) {
                long z = nbr(P, y, CXQ[q], CYQ[q], CZQ[q]);
                if (!(ft[z] & (FL_LIQ | FL_IF))) continue;
                double fz[NQ], rz, uz[3];
                for (int p = 0; p < NQ; ++p) fz[p] = fout[(long)p * N + z];
                moments(fz, &rz, uz);
                rs += rz;
                us[0] += uz[0];
                us[1] += uz[1];
                us[2] += uz[2];
                ++cnt;
            }
            double rb = rs / cnt, ub[3] = {us[0] / cnt, us[1] / cnt, us[2] / cnt};
            for (int q = 0; q < NQ; ++q) fout[(long)q * N + y] = feq(q, rb, ub);
            rho[y] = rb;
            mnew[y] = 0;
        } else if (newif[y] == 2) {
            mnew[y] = rho[y];
        }
    }
    /* excess mass, shared by the interface cells after conversion: equally
     * (reading O7), or weighted by the interface normal (reading K1, after
     * Koerner et al.: a filled cell gives to the gas side, weight
     * max(0, -n.c_q), an emptied one to the liquid side, max(0, n.c_q), n the
     * PLIC normal of the cell at t (pointing into the liquid), c_q the
     * lattice vector to the receiver; equal shares if every weight is 0) */
    for (long x = 0; x < N; ++x) {
        if (!conv[x]) continue;
        double mex;
        if (conv[x] == 1) {
            mex = mnew[x] - rho[x];
            mnew[x] = rho[x];
        } else {
            mex = mnew[x];
            mnew[x] = 0;
        }
        int n = 0;
        double W = 0, wq[NQ];
        const double *nx4 = normal4 + 4 * x;
        const double sgn = conv[x] == 1 ? -1.0 : 1.0;
        for (int q = 1; q < NQ; ++q) {
            long y = nbr(P, x, CXQ[q], CYQ[q], CZQ[q]);
            wq[q] = 0;
            if (((ft[y] & FL_IF) && !conv[y]) || newif[y]) {
                ++n;
                double nc = nx4[0] * CXQ[q] + nx4[1] * CYQ[q] + nx4[2] * CZQ[q];
                wq[q] = fmax(0.0, sgn * nc);
                W += wq[q];
            }
        }
        if (n == 0) {
            *lost += mex;
            continue;
        }
        for (int q = 1; q < NQ; ++q) {
            long y = nbr(P, x, CXQ[q], CYQ[q], CZQ[q]);
            if (!(((ft[y] & FL_IF) && !conv[y]) || newif[y])) continue;
            if (P->excess_rule == 1 && W > 0) mnew[y] += mex * (wq[q] / W);
            else mnew[y] += mex / n;
        }
    }
    for (long x = 0; x < N; ++x) {
        uint8_t t = ft[x];
        if (conv[x] == 1) { t = FL_LIQ; counts[3]++; }
        else if (conv[x] == 2) { t = FL_GAS; counts[4]++; }
        else if (newif[x]) { t = FL_IF; counts[newif[x] == 1 ? 5 : 6]++; }
        flags[x] = t;
        if (t & FL_IF) {
            mass[x] = mnew[x];
            phi[x] = mnew[x] / rho[x];
        } else if (t & FL_LIQ) {
            mass[x] = rho[x];
            phi[x] = 1.0;
        } else if (t & FL_GAS) {
            mass[x] = 0;
            phi[x] = 0;
        }
    }
    for (long x = 0; x < N; ++x) {
        if (flags[x] & FL_LIQ) counts[0]++;
        if (flags[x] & FL_GAS) counts[2]++;
        int hl = 0, hg = 0;
        for (int q = 1; q < NQ; ++q) {
            uint8_t t = flags[nbr(P, x, CXQ[q], CYQ[q], CZQ[q])];
            hl |= (t & FL_LIQ) != 0;
            hg |= (t & FL_GAS) != 0;
        }
        if (flags[x] & FL_IF) {
            counts[1]++;
            if (!hl || !hg) counts[7]++;
        }
        if ((flags[x] & FL_LIQ) && hg) counts[8]++;
    }
    free(ft);
    free(conv);
    free(newif);
    free(mnew);
}

/* ------------------------------------------------------------------------ */
/* initial state (Sec. III.A: fill levels by sub-division of each cell)      */

static int inside(const orc_geom *G, double px, double py, double pz) {
    int in = 0;
    double dx = px - G->c[0], dy = py - G->c[1], dz = pz - G->c[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    switch (G->kind) {
    case 0: in = r2 <= G->R * G->R; break;
    case 1: {
        double r = sqrt(r2);
        if (r == 0) { in = 1; break; }
        double mu = dz / r;
        in = r <= G->R * (1.0 + G->eps2 * (1.5 * mu * mu - 0.5));
        break;
    }
    case 2: in = (r2 <= G->R * G->R) && (pz >= G->zw); break;
    case 3: {
        double ex = px - G->c2[0], ey = py - G->c2[1], ez = pz - G->c2[2];
        in = (r2 <= G->R * G->R) || (ex * ex + ey * ey + ez * ez <= G->R2 * G->R2);
        break;
    }
    case 4: {
        const double tp = 6.283185307179586;
        in = pz < G->h0 + G->amp * sin(tp * px / G->wavelength) * sin(tp * py / G->wavelength);
        break;
    }
    case 5: in = G->n[0] * px + G->n[1] * py + G->n[2] * pz <= G->d; break;
    }
    return G->invert ? !in : in;
}

/* fill level of one cell (centre (x,y,z), extent +-1/2): the fraction of the
 * sub^3 points x + (s + 1/2)/sub - 1/2 inside the shape (Sec. III.A). */
double orc_fill_cell(const orc_geom *G, int x, int y, int z) {
    int S = G->sub, cnt = 0;
    for (int sz = 0; sz < S; ++sz)
        for (int sy = 0; sy < S; ++sy)
            for (int sx = 0; sx < S; ++sx)
                cnt += inside(G, x + (sx + 0.5) / S - 0.5, y + (sy + 0.5) / S - 0.5, z + (sz + 0.5) / S - 0.5);
    return (double)cnt / ((double)S * S * S);
}

/* whole field; cells are sampled one by one (no shortcut) */
void orc_fill(const orc_geom *G, int nx, int ny, int nz, double *phi) {
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) phi[x + (long)nx * (y + (long)ny * z)] = orc_fill_cell(G, x, y, z);
}

/* fill levels of a list of cells (for sampled checks on large grids) */
void orc_fill_list(const orc_geom *G, int nx, int ny, long n, const long *idx, double *out) {
    for (long k = 0; k < n; ++k) {
        long i = idx[k];
        int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / ((long)nx * ny));
        out[k] = orc_fill_cell(G, x, y, z);
    }
}

/* Cell types from fill levels (Sec. II: only interface cells have 0 < phi < 1;
 * an interface cell has liquid and gas neighbours): obstacle cells keep their
 * type; phi <= 0 gas, phi >= 1 liquid, else interface; then every liquid cell
 * with a gas D3Q19 neighbour becomes interface, so that no liquid cell touches
 * a gas cell.  f = feq(1, 0) = w_q, m = phi (rho = 1). */
void orc_init_state(const orc_params *P, const uint8_t *obstacle, double *phi, uint8_t *flags, double *f,
                    double *mass) {
    long N = ncell(P);
    for (long i = 0; i < N; ++i) {
        if (obstacle[i]) flags[i] = FL_OBS;
        else if (phi[i] <= 0) flags[i] = FL_GAS;
        else if (phi[i] >= 1) flags[i] = FL_LIQ;
        else flags[i] = FL_IF;
    }
    for (long i = 0; i < N; ++i) {
        if (!(flags[i] & FL_LIQ)) continue;
        for (int q = 1; q < NQ; ++q)
            if (flags[nbr(P, i, CXQ[q], CYQ[q], CZQ[q])] == FL_GAS) {
                flags[i] = FL_IF | 0x80; /* mark: was liquid */
                break;
            }
    }
    for (long i = 0; i < N; ++i) {
        flags[i] &= FL_TYPE;
        if (flags[i] & FL_OBS) phi[i] = 0;
        if (flags[i] & FL_GAS) phi[i] = 0;
        if (flags[i] & FL_LIQ) phi[i] = 1;
        mass[i] = (flags[i] & (FL_LIQ | FL_IF)) ? phi[i] : 0;
        for (int q = 0; q < NQ; ++q) f[(long)q * N + i] = w_q(q);
    }
}

/* total mass: sum of m over interface cells plus sum of rho over liquid cells */
double orc_mass(const orc_params *P, const uint8_t *flags, const double *f, const double *mass) {
    long N = ncell(P);
    double M = 0;
    for (long i = 0; i < N; ++i) {
        if (flags[i] & FL_IF) M += mass[i];
        else if (flags[i] & FL_LIQ) {
            double r = 0;
            for (int q = 0; q < NQ; ++q) r += f[(long)q * N + i];
            M += r;
        }
    }
    return M;
}
