/*
 * lbm_oracle.c -- plain, slow, FP64 CPU oracle for the lattice Boltzmann hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or calls this
 * file; only the test suite, the smoke check and the CPU-baseline leg of the benchmark load
 * it.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (waLBerla paper, Sec. 5.1, lattice Boltzmann method):
 *   - Eq. 1: density and momentum density are the zeroth and first moments of the PDFs.
 *   - Eq. 2: f_i(x + c_i, t + 1) = f_i(x, t) + Omega_i(f(x, t)): collide, then push each
 *     post-collision PDF to the neighbour it points at.
 *   - Eq. 3 with the special relaxation matrices named right after it: SRT (one rate) and
 *     TRT (one rate for the even part, one for the odd part of each direction pair); and
 *     Eq. 3 itself (MRT) with a stated moment matrix and one rate per group of moments;
 *     and the cumulant collision the same section names (D3Q27: cumulants relaxed towards
 *     their equilibria, one rate per group).
 *   - Sec. 5.1.1, body-force paragraph: a constant body force drives periodic set-ups; the
 *     force model is Guo et al. (the paper cites it), split into even/odd parts under TRT.
 *   - Sec. 5.1.1, boundary paragraph: no-slip, velocity and pressure boundaries.  The paper
 *     cites Ginzburg 2008 for them; the oracle takes halfway bounce-back (no-slip),
 *     bounce-back with a wall-velocity term (velocity) and anti-bounce-back (pressure).
 *   - Sec. 4.4: boundary handling by iterating over all cells and reading a per-cell flag
 *     field, the simple method the paper describes first.  The CUDA path uses the
 *     per-kind link lists instead.
 * The paper fixes none of the constants of these operators; the reading adopted for each
 * one is stated next to the code below.
 *
 * State convention: the oracle's state is the post-collision field f*(x, t) at fluid cells
 * (the right-hand side of Eq. 2).  Arrays are f[i][z][y][x] with no ghost layer; the global
 * domain has nx*ny*nz cells and knows nothing about blocks.
 *
 * Floating point: every operation is IEEE double, evaluated in source order (the build
 * passes -ffp-contract=off so x86-64 and aarch64 give the same bits).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* cell / face kinds (flag field values) */
#define ORC_FLUID 0
#define ORC_NOSLIP 1
#define ORC_VELOCITY 2
#define ORC_PRESSURE 3
#define ORC_PERIODIC 4 /* face kind only */
#define ORC_ZOUHE_VELOCITY 5 /* face kind only: wet-node velocity boundary (Zou & He) */
#define ORC_ZOUHE_PRESSURE 6 /* face kind only: wet-node pressure boundary (Zou & He) */

#define ORC_SRT 0
#define ORC_TRT 1
#define ORC_MRT 2
#define ORC_CUMULANT 3

#define QMAX 27

typedef struct {
    int32_t q;            /* 19 or 27 */
    int32_t collision;    /* ORC_SRT, ORC_TRT, ORC_MRT or ORC_CUMULANT */
    int32_t nx, ny, nz;   /* global domain size in cells */
    int32_t periodic[3];  /* non-zero: axis is periodic */
    int32_t face_kind[6]; /* kind of the region outside face (axis, side) = index 2*axis+side */
    double omega;         /* SRT: omega = 1/tau; TRT: omega_plus */
    double magic_lambda;  /* TRT: Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) */
    double force[3];      /* constant body force per cell, lattice units */
    double face_u[6][3];  /* wall velocity of a velocity face */
    double face_rho[6];   /* wall density of a velocity face / pressure of a pressure face */
    double mrt_s[7];      /* MRT: rates of the row groups 1..7 (momentum, shear, bulk, third,
                             fourth, fifth, sixth order; see the MRT section below) */
    double cum_s[9];      /* cumulant: rates of the groups 2..10 (group 1, shear, takes omega;
                             see the cumulant section below) */
} orc_params;

/* ---------------------------------------------------------------------------------------
 * Lattice.  The paper names D3Q19 and D3Q27 (Sec. 5.1.1) but prints no table.  The oracle
 * enumerates the velocity set from its definition: all c in {-1,0,1}^3 with |c|^2 <= 2
 * (D3Q19) or <= 3 (D3Q27), ordered by |c|^2 first; within |c|^2 = 1 the order is
 * +x,-x,+y,-y,+z,-z; within |c|^2 = 2 and 3 it is lexicographic in (cx,cy,cz).  Weights are
 * the standard ones that make the lattice isotropic to fourth order with c_s^2 = 1/3:
 * D3Q19 1/3, 1/18, 1/36 and D3Q27 8/27, 2/27, 1/54, 1/216 by |c|^2 = 0,1,2,3.
 * ------------------------------------------------------------------------------------- */
int orc_lattice(int q, int *c, double *w, int *opp)
{
    if (q != 19 && q != 27) return -1;
    int maxsq = (q == 19) ? 2 : 3;
    int n = 0;
    /* |c|^2 = 0 */
    c[0] = c[1] = c[2] = 0;
    n = 1;
    /* |c|^2 = 1: one axis at a time, positive before negative */
    for (int a = 0; a < 3; ++a) {
        for (int s = 0; s < 2; ++s) {
            c[3 * n + 0] = c[3 * n + 1] = c[3 * n + 2] = 0;
            c[3 * n + a] = s == 0 ? 1 : -1;
            ++n;
        }
    }
    /* |c|^2 = 2, then 3: lexicographic */
    for (int sq = 2; sq <= maxsq; ++sq) {
        for (int cx = -1; cx <= 1; ++cx)
            for (int cy = -1; cy <= 1; ++cy)
                for (int cz = -1; cz <= 1; ++cz) {
                    if (cx * cx + cy * cy + cz * cz != sq) continue;
                    c[3 * n + 0] = cx;
                    c[3 * n + 1] = cy;
                    c[3 * n + 2] = cz;
                    ++n;
                }
    }
    if (n != q) return -2;
    for (int i = 0; i < q; ++i) {
        int sq = c[3 * i] * c[3 * i] + c[3 * i + 1] * c[3 * i + 1] + c[3 * i + 2] * c[3 * i + 2];
        if (q == 19)
            w[i] = sq == 0 ? 1.0 / 3.0 : (sq == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        else
            w[i] = sq == 0 ? 8.0 / 27.0 : (sq == 1 ? 2.0 / 27.0 : (sq == 2 ? 1.0 / 54.0 : 1.0 / 216.0));
        opp[i] = -1;
        for (int j = 0; j < q; ++j)
            if (c[3 * j] == -c[3 * i] && c[3 * j + 1] == -c[3 * i + 1] && c[3 * j + 2] == -c[3 * i + 2])
                opp[i] = j;
        if (opp[i] < 0) return -3;
    }
    return 0;
}

typedef struct {
    int q;
    int c[3 * QMAX];
    double w[QMAX];
    int opp[QMAX];
    double M[QMAX * QMAX];    /* MRT moment matrix, row k = moment k, M[k * q + i] */
    double Minv[QMAX * QMAX]; /* its inverse, Minv[i * q + k] */
    int group[QMAX];          /* row group of moment k (0 mass, 1..7 as mrt_s) */
} lattice_t;

static int mrt_matrix(lattice_t *L);

static void cumulant_table(void);

static int get_lattice(int q, lattice_t *L)
{
    L->q = q;
    int r = orc_lattice(q, L->c, L->w, L->opp);
    if (r != 0) return r;
    if (q == 27) cumulant_table();
    return mrt_matrix(L);
}

/* ---------------------------------------------------------------------------------------
 * MRT moment space (Eq. 3: Omega = -M^-1 S (M f - m_eq), M invertible, S diagonal).  The
 * paper cites d'Humieres et al. 2002 for the method and fixes neither M nor S.  Reading:
 * the rows of M are polynomials in c_i, each of one parity, taken in this order and grouped
 * by degree (group number in brackets):
 *   [0] 1;  [1] cx, cy, cz;
 *   [2] cx cy, cx cz, cy cz, 2cx^2 - cy^2 - cz^2, cy^2 - cz^2 (shear);  [3] |c|^2 (bulk);
 *   [4] cx(cy^2 + cz^2), cx(cy^2 - cz^2), cy(cx^2 + cz^2), cy(cx^2 - cz^2),
 *       cz(cx^2 + cy^2), cz(cx^2 - cy^2), and for D3Q27 cx cy cz;
 *   [5] cx^2 cy^2, cx^2 cz^2, cy^2 cz^2, and for D3Q27 cx^2 cy cz, cy^2 cx cz, cz^2 cx cy;
 *   [6] (D3Q27) cx^2 cy^2 cz, cx^2 cz^2 cy, cy^2 cz^2 cx;  [7] (D3Q27) cx^2 cy^2 cz^2;
 * evaluated at the lattice velocities and orthogonalised one after the other by Gram-Schmidt
 * under the weighted product <a, b> = sum_i w_i a_i b_i.  Every row is then orthogonal to all
 * rows before it, so a group's rows span the polynomials of its degree class with everything
 * of lower classes removed, and relaxing a group with one rate does not depend on how the
 * rows within it are chosen.  S holds one rate per group: mass (group 0) is conserved,
 * groups 1..7 take mrt_s[0..6].  The Guo source enters moment space with the factor
 * (1 - s/2) of its own moment's rate.  M^-1 is computed by Gauss-Jordan elimination, not
 * from the orthogonality.
 * ------------------------------------------------------------------------------------- */
static double mrt_raw(int k27, const int *c, int *group)
{
    const double x = c[0], y = c[1], z = c[2];
    const double xx = x * x, yy = y * y, zz = z * z;
    switch (k27) {
        case 0: *group = 0; return 1.0;
        case 1: *group = 1; return x;
        case 2: *group = 1; return y;
        case 3: *group = 1; return z;
        case 4: *group = 2; return x * y;
        case 5: *group = 2; return x * z;
        case 6: *group = 2; return y * z;
        case 7: *group = 2; return 2.0 * xx - yy - zz;
        case 8: *group = 2; return yy - zz;
        case 9: *group = 3; return xx + yy + zz;
        case 10: *group = 4; return x * (yy + zz);
        case 11: *group = 4; return x * (yy - zz);
        case 12: *group = 4; return y * (xx + zz);
        case 13: *group = 4; return y * (xx - zz);
        case 14: *group = 4; return z * (xx + yy);
        case 15: *group = 4; return z * (xx - yy);
        case 16: *group = 4; return x * y * z;
        case 17: *group = 5; return xx * yy;
        case 18: *group = 5; return xx * zz;
        case 19: *group = 5; return yy * zz;
        case 20: *group = 5; return xx * y * z;
        case 21: *group = 5; return yy * x * z;
        case 22: *group = 5; return zz * x * y;
        case 23: *group = 6; return xx * yy * z;
        case 24: *group = 6; return xx * zz * y;
        case 25: *group = 6; return yy * zz * x;
        default: *group = 7; return xx * yy * zz;
    }
}

static int mrt_matrix(lattice_t *L)
{
    const int q = L->q;
    /* D3Q19 takes the rows 0..15 and 17..19 of the D3Q27 list */
    static const int rows19[19] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 17, 18, 19};
    for (int k = 0; k < q; ++k) {
        const int r = q == 19 ? rows19[k] : k;
        for (int i = 0; i < q; ++i) L->M[k * q + i] = mrt_raw(r, L->c + 3 * i, &L->group[k]);
    }
    /* Gram-Schmidt under the weighted product, rows in order */
    for (int k = 0; k < q; ++k) {
        for (int j = 0; j < k; ++j) {
            double num = 0.0, den = 0.0;
            for (int i = 0; i < q; ++i) {
                num += L->w[i] * L->M[k * q + i] * L->M[j * q + i];
                den += L->w[i] * L->M[j * q + i] * L->M[j * q + i];
            }
            const double a = num / den;
            for (int i = 0; i < q; ++i) L->M[k * q + i] -= a * L->M[j * q + i];
        }
        double nn = 0.0;
        for (int i = 0; i < q; ++i) nn += L->w[i] * L->M[k * q + i] * L->M[k * q + i];
        if (!(nn > 1e-12)) return -4; /* the rows are not independent on this lattice */
    }
    /* inverse by Gauss-Jordan elimination with partial pivoting on [M | I] */
    double A[QMAX][2 * QMAX];
    for (int r = 0; r < q; ++r)
        for (int j = 0; j < 2 * q; ++j) A[r][j] = j < q ? L->M[r * q + j] : (j - q == r ? 1.0 : 0.0);
    for (int col = 0; col < q; ++col) {
        int piv = col;
        for (int r = col + 1; r < q; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (fabs(A[piv][col]) < 1e-14) return -5;
        if (piv != col)
            for (int j = 0; j < 2 * q; ++j) {
                double t = A[col][j];
                A[col][j] = A[piv][j];
                A[piv][j] = t;
            }
        const double d = A[col][col];
        for (int j = 0; j < 2 * q; ++j) A[col][j] /= d;
        for (int r = 0; r < q; ++r) {
            if (r == col) continue;
            const double a = A[r][col];
            if (a == 0.0) continue;
            for (int j = 0; j < 2 * q; ++j) A[r][j] -= a * A[col][j];
        }
    }
    for (int i = 0; i < q; ++i)
        for (int k = 0; k < q; ++k) L->Minv[i * q + k] = A[i][q + k];
    return 0;
}

/* The moment matrix, its inverse and the row groups (for the tests). */
int orc_mrt_matrix(int q, double *M, double *Minv, int *group)
{
    lattice_t L;
    int r = get_lattice(q, &L);
    if (r != 0) return r;
    memcpy(M, L.M, sizeof(double) * q * q);
    memcpy(Minv, L.Minv, sizeof(double) * q * q);
    memcpy(group, L.group, sizeof(int) * q);
    return 0;
}

/* TRT: the second rate follows from the "magic" parameter
 *   Lambda = (1/omega+ - 1/2) (1/omega- - 1/2)        (Ginzburg 2008, cited for TRT). */
double orc_omega_minus(double omega_plus, double magic_lambda)
{
    double lp = 1.0 / omega_plus - 0.5;
    return 1.0 / (magic_lambda / lp + 0.5);
}

/* Second-order polynomial equilibrium, compressible form (rho multiplies every term):
 *   f_eq_i = w_i rho [1 + 3 c_i.u + 9/2 (c_i.u)^2 - 3/2 u.u].
 * Same form for D3Q19 and D3Q27 (the paper does not fix it; this is the standard choice). */
static void equilibrium(const lattice_t *L, double rho, const double u[3], double *feq)
{
    double usq = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < L->q; ++i) {
        double cu = L->c[3 * i] * u[0] + L->c[3 * i + 1] * u[1] + L->c[3 * i + 2] * u[2];
        feq[i] = L->w[i] * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
    }
}

void orc_equilibrium(int q, double rho, const double *u, double *feq)
{
    lattice_t L;
    if (get_lattice(q, &L) != 0) return;
    equilibrium(&L, rho, u, feq);
}

/* Eq. 1 plus the Guo half-force shift:  rho = sum f,  rho u = sum c f + F/2. */
static void moments_pre(const lattice_t *L, const double *f, const double F[3], double *rho, double u[3])
{
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i) {
        r += f[i];
        j[0] += L->c[3 * i] * f[i];
        j[1] += L->c[3 * i + 1] * f[i];
        j[2] += L->c[3 * i + 2] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] + 0.5 * F[a]) / r;
}

/* Moments of a post-collision state: the collision adds F to sum c f, so the physical
 * velocity of the same time level is (sum c f* - F/2) / rho.  Used for output and for the
 * pressure boundary's u_b. */
static void moments_post(const lattice_t *L, const double *f, const double F[3], double *rho, double u[3])
{
    double r = 0.0, j[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < L->q; ++i) {
        r += f[i];
        j[0] += L->c[3 * i] * f[i];
        j[1] += L->c[3 * i + 1] * f[i];
        j[2] += L->c[3 * i + 2] * f[i];
    }
    *rho = r;
    for (int a = 0; a < 3; ++a) u[a] = (j[a] - 0.5 * F[a]) / r;
}

/* ---------------------------------------------------------------------------------------
 * Locally varying relaxation (Sec. 5.1.1: methods that vary the relaxation rate per cell
 * from a local fluid property, e.g. turbulence models after Yu et al. 2005, cited there;
 * waLBerla reads such rates from a separate field).  The closure gives the cell's omega+
 * from its pre-collision state; omega- follows from the same Lambda.
 *   Pi_neq_ab = sum_i c_ia c_ib f_i - rho (delta_ab / 3 + u_a u_b)   (non-equilibrium stress)
 *   kind 1, Smagorinsky with constant cs (grid spacing 1): the total relaxation time tau
 *   solves nu_t = (tau - tau0)/3 = cs^2 |S| with |S| = 3 sqrt(2 Pi:Pi) / (2 rho tau), i.e.
 *       tau = ( tau0 + sqrt(tau0^2 + 18 cs^2 sqrt(2 Pi:Pi) / rho) ) / 2
 *   kind 2, MLP: features (rho - 1) s_rho and s_pi Pi_neq (xx, yy, zz, xy, xz, yz), two
 *   hidden layers of 32 SiLU units, one output y; tau = tau0 + s_tau softplus(y).  The
 *   network is the model as deployed: its three weight matrices are BF16 numbers (the
 *   packed FP32 weights rounded to nearest even), its biases the packed FP32 values;
 *   features, sums, SiLU and hidden activations are exact FP64 (no rounding of features or
 *   activations).  Packed parameters (float): W1[32][7], b1[32], W2[32][32], b2[32],
 *   w3[32], b3, s_rho, s_pi, s_tau.
 * ------------------------------------------------------------------------------------- */
typedef struct {
    int32_t kind; /* 0 none, 1 Smagorinsky, 2 MLP */
    int32_t pad;
    double cs;
    const float *mlp;
} orc_closure;

#define MLP_H 32
#define MLP_IN 7

static double bf16(double v)
{
    float f = (float)v;
    uint32_t b;
    memcpy(&b, &f, 4);
    b += 0x7fffu + ((b >> 16) & 1u);
    b &= 0xffff0000u;
    memcpy(&f, &b, 4);
    return (double)f;
}

static double silu(double z) { return z / (1.0 + exp(-z)); }

static double softplus(double y) { return y > 30.0 ? y : log1p(exp(y)); }

/* Non-equilibrium stress of a pre-collision state (rho, u with the half-force shift). */
static void pi_neq(const lattice_t *L, const double *f, double rho, const double u[3], double pi[6])
{
    double m[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < L->q; ++i) {
        double cx = L->c[3 * i], cy = L->c[3 * i + 1], cz = L->c[3 * i + 2];
        m[0] += cx * cx * f[i];
        m[1] += cy * cy * f[i];
        m[2] += cz * cz * f[i];
        m[3] += cx * cy * f[i];
        m[4] += cx * cz * f[i];
        m[5] += cy * cz * f[i];
    }
    pi[0] = m[0] - rho * (1.0 / 3.0 + u[0] * u[0]);
    pi[1] = m[1] - rho * (1.0 / 3.0 + u[1] * u[1]);
    pi[2] = m[2] - rho * (1.0 / 3.0 + u[2] * u[2]);
    pi[3] = m[3] - rho * u[0] * u[1];
    pi[4] = m[4] - rho * u[0] * u[2];
    pi[5] = m[5] - rho * u[1] * u[2];
}

/* MLP output y for one cell's features: BF16 weights, everything else exact FP64. */
static double mlp_y(const float *P, const double feat[MLP_IN])
{
    const float *W1 = P, *b1 = P + MLP_H * MLP_IN, *W2 = b1 + MLP_H, *b2 = W2 + MLP_H * MLP_H, *w3 = b2 + MLP_H,
                *b3 = w3 + MLP_H;
    double h1[MLP_H], h2[MLP_H];
    for (int j = 0; j < MLP_H; ++j) {
        double z = b1[j];
        for (int k = 0; k < MLP_IN; ++k) z += bf16(W1[j * MLP_IN + k]) * feat[k];
        h1[j] = silu(z);
    }
    for (int j = 0; j < MLP_H; ++j) {
        double z = b2[j];
        for (int k = 0; k < MLP_H; ++k) z += bf16(W2[j * MLP_H + k]) * h1[k];
        h2[j] = silu(z);
    }
    double y = b3[0];
    for (int k = 0; k < MLP_H; ++k) y += bf16(w3[k]) * h2[k];
    return y;
}

/* omega+ of a cell under the closure (p->omega is the base rate 1/tau0). */
static double closure_omega(const lattice_t *L, const orc_params *p, const orc_closure *cl, const double *f,
                            double rho, const double u[3])
{
    if (!cl || cl->kind == 0) return p->omega;
    const double tau0 = 1.0 / p->omega;
    double pi[6];
    pi_neq(L, f, rho, u, pi);
    if (cl->kind == 1) {
        double q = pi[0] * pi[0] + pi[1] * pi[1] + pi[2] * pi[2] + 2.0 * (pi[3] * pi[3] + pi[4] * pi[4] + pi[5] * pi[5]);
        double tau = 0.5 * (tau0 + sqrt(tau0 * tau0 + 18.0 * cl->cs * cl->cs * sqrt(2.0 * q) / rho));
        return 1.0 / tau;
    }
    const float *P = cl->mlp;
    const float *tail = P + MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1;
    const double s_rho = tail[0], s_pi = tail[1], s_tau = tail[2];
    double feat[MLP_IN] = {(rho - 1.0) * s_rho, pi[0] * s_pi, pi[1] * s_pi, pi[2] * s_pi,
                           pi[3] * s_pi,        pi[4] * s_pi, pi[5] * s_pi};
    return 1.0 / (tau0 + s_tau * softplus(mlp_y(P, feat)));
}

/* Collision operator Omega of Eq. 2, SRT or TRT (Eq. 3 with special S), with Guo forcing:
 *   S_i = w_i [3 (c_i - u) + 9 (c_i.u) c_i] . F
 *   SRT: f*_i = f_i - w (f_i - feq_i) + (1 - w/2) S_i
 *   TRT: g+- = (g_i +- g_opp(i)) / 2 for g in {f, feq, S};
 *        f*_i = f_i - w+ (f+ - feq+) - w- (f- - feq-) + (1 - w+/2) S+ + (1 - w-/2) S-.     */
static void collide_cumulant(const lattice_t *L, const orc_params *p, const double *f, double *fout);

static void collide(const lattice_t *L, const orc_params *p, const orc_closure *cl, const double *f, double *fout)
{
    if (p->collision == ORC_CUMULANT) {
        collide_cumulant(L, p, f, fout);
        return;
    }
    const double *F = p->force;
    double rho, u[3];
    moments_pre(L, f, F, &rho, u);
    const double om = closure_omega(L, p, cl, f, rho, u);
    double feq[QMAX], S[QMAX];
    equilibrium(L, rho, u, feq);
    for (int i = 0; i < L->q; ++i) {
        double cx = L->c[3 * i], cy = L->c[3 * i + 1], cz = L->c[3 * i + 2];
        double cu = cx * u[0] + cy * u[1] + cz * u[2];
        double ax = 3.0 * (cx - u[0]) + 9.0 * cu * cx;
        double ay = 3.0 * (cy - u[1]) + 9.0 * cu * cy;
        double az = 3.0 * (cz - u[2]) + 9.0 * cu * cz;
        S[i] = L->w[i] * (ax * F[0] + ay * F[1] + az * F[2]);
    }
    if (p->collision == ORC_SRT) {
        double w = om;
        for (int i = 0; i < L->q; ++i) fout[i] = f[i] - w * (f[i] - feq[i]) + (1.0 - 0.5 * w) * S[i];
    } else if (p->collision == ORC_MRT) {
        /* Eq. 3 in moment space: m* = m - S (m - meq) + (I - S/2) g, f* = M^-1 m* */
        const int q = L->q;
        double ms[QMAX];
        for (int k = 0; k < q; ++k) {
            double m = 0.0, me = 0.0, g = 0.0;
            for (int i = 0; i < q; ++i) {
                m += L->M[k * q + i] * f[i];
                me += L->M[k * q + i] * feq[i];
                g += L->M[k * q + i] * S[i];
            }
            const double s = L->group[k] == 0 ? 0.0 : p->mrt_s[L->group[k] - 1];
            ms[k] = m - s * (m - me) + (1.0 - 0.5 * s) * g;
        }
        for (int i = 0; i < q; ++i) {
            double v = 0.0;
            for (int k = 0; k < q; ++k) v += L->Minv[i * q + k] * ms[k];
            fout[i] = v;
        }
    } else {
        double wp = om;
        double wm = orc_omega_minus(wp, p->magic_lambda);
        for (int i = 0; i < L->q; ++i) {
            int o = L->opp[i];
            double fp = 0.5 * (f[i] + f[o]), fm = 0.5 * (f[i] - f[o]);
            double ep = 0.5 * (feq[i] + feq[o]), em = 0.5 * (feq[i] - feq[o]);
            double sp = 0.5 * (S[i] + S[o]), sm = 0.5 * (S[i] - S[o]);
            fout[i] = f[i] - wp * (fp - ep) - wm * (fm - em) + (1.0 - 0.5 * wp) * sp + (1.0 - 0.5 * wm) * sm;
        }
    }
}

/* ---------------------------------------------------------------------------------------
 * Cumulant collision (Sec. 5.1.1: cumulants instead of moments are relaxed towards their
 * equilibria; the paper cites Geier et al. 2015 for the method and fixes none of its
 * details).  D3Q27 only: its velocities are all of {-1,0,1}^3, so the 27 central moments
 * kappa_abc with a, b, c in {0, 1, 2} determine the 27 populations.
 *   rho = sum f,  u = (sum c f + F/2) / rho                          (the Guo half-force shift)
 *   kappa_abc = sum_i f_i (c_ix - u_x)^a (c_iy - u_y)^b (c_iz - u_z)^c          (definition)
 *   cumulants of order >= 2, density-scaled: C_abc = rho k_abc with k from mu = kappa / rho
 *   by the moment-cumulant formula over the set partitions pi of the multiset of a x's,
 *   b y's and c z's,
 *       k = sum_pi (-1)^(|pi| - 1) (|pi| - 1)! prod_{B in pi} mu_B ,
 *   where mu_B is the central moment of the block's variables.  Reading: the first central
 *   moments are taken as zero in this formula (partitions with a one-element block drop
 *   out), i.e. the cumulants of a distribution centred on u.  Without a body force that is
 *   exact (u is the mean); with one, the populations' mean is u - F/(2 rho) and the
 *   collision moves that first-order part separately: kappa_100 = -F_x/2 before it and
 *   +F_x/2 after it, so that sum c f* = sum c f + F.
 *   Relaxation, one rate per group (group 1 = omega, groups 2..10 = cum_s[0..8]); every
 *   cumulant of order >= 3 has equilibrium 0, the second-order ones rho/3 on the diagonal:
 *     [1] C_110, C_101, C_011 and C_200 - C_020, C_200 - C_002                 (shear)
 *     [2] C_200 + C_020 + C_002, towards rho                                   (bulk)
 *     [3] C_120 + C_102, C_210 + C_012, C_201 + C_021
 *     [4] C_120 - C_102, C_210 - C_012, C_201 - C_021
 *     [5] C_111
 *     [6] C_220 - 2 C_202 + C_022, C_220 + C_202 - 2 C_022
 *     [7] C_220 + C_202 + C_022
 *     [8] C_211, C_121, C_112
 *     [9] C_221, C_212, C_122
 *    [10] C_222
 *   each combination g going to g - s (g - g_eq).  Back: mu* from C* / rho by the same
 *   formula solved for its one-block term, in order of increasing order (every other term
 *   has blocks of lower order, already known); kappa* = rho mu*; f* from kappa* by
 *   inverting the map f -> kappa, which is the tensor product of one 3 x 3 map per axis,
 *   (p_-, p_0, p_+) -> (sum p, sum p d, sum p d^2) with d = c - u_axis, inverted in closed
 *   form: A = m1 + u m0, B = m2 + 2 u m1 + u^2 m0, p_0 = m0 - B, p_+- = (B +- A) / 2.
 * ------------------------------------------------------------------------------------- */
#define CUM_MAXT 64

typedef struct {
    int nterm[27];             /* terms of cumulant (a, b, c), index a + 3 b + 9 c */
    double coef[27][CUM_MAXT]; /* (-1)^(m - 1) (m - 1)! for a partition into m blocks */
    int nblk[27][CUM_MAXT];
    int blk[27][CUM_MAXT][3];  /* central-moment index of each block */
} cum_table_t;

static cum_table_t g_cum;
static int g_cum_ready = 0;

/* all set partitions of the n variables var[0..n-1] (0 = x, 1 = y, 2 = z) by restricted
 * growth strings: element j joins one of the blocks used so far or opens a new one */
static void cum_partitions(int k, const int *var, int n, int *blockof, int j, int nb)
{
    if (j == n) {
        int cnt[6][3];
        memset(cnt, 0, sizeof cnt);
        for (int e = 0; e < n; ++e) cnt[blockof[e]][var[e]]++;
        for (int b = 0; b < nb; ++b)
            if (cnt[b][0] + cnt[b][1] + cnt[b][2] == 1) return; /* a one-element block: mu = 0 */
        int t = g_cum.nterm[k]++;
        double fact = 1.0;
        for (int m = 2; m < nb; ++m) fact *= m;
        g_cum.coef[k][t] = (nb % 2 == 1 ? 1.0 : -1.0) * fact;
        g_cum.nblk[k][t] = nb;
        for (int b = 0; b < nb; ++b) g_cum.blk[k][t][b] = cnt[b][0] + 3 * cnt[b][1] + 9 * cnt[b][2];
        return;
    }
    for (int b = 0; b <= nb && b < 6; ++b) {
        blockof[j] = b;
        cum_partitions(k, var, n, blockof, j + 1, b == nb ? nb + 1 : nb);
    }
}

static void cumulant_table(void)
{
    if (g_cum_ready) return;
    memset(&g_cum, 0, sizeof g_cum);
    for (int k = 0; k < 27; ++k) {
        int a = k % 3, b = (k / 3) % 3, c = k / 9, var[6], n = 0, blockof[6];
        for (int e = 0; e < a; ++e) var[n++] = 0;
        for (int e = 0; e < b; ++e) var[n++] = 1;
        for (int e = 0; e < c; ++e) var[n++] = 2;
        if (n >= 2) cum_partitions(k, var, n, blockof, 0, 0);
    }
    g_cum_ready = 1;
}

static int cum_order(int k) { return k % 3 + (k / 3) % 3 + k / 9; }

/* rho, u, and the density-scaled cumulants C[27] of f (C[0] = rho, C[first order] = the
 * central first moments kappa_100, kappa_010, kappa_001) */
static void cumulants(const lattice_t *L, const double *f, const double F[3], double *rho, double u[3],
                      double *C)
{
    moments_pre(L, f, F, rho, u);
    double mu[27];
    for (int k = 0; k < 27; ++k) {
        int a = k % 3, b = (k / 3) % 3, c = k / 9;
        double m = 0.0;
        for (int i = 0; i < 27; ++i) {
            double dx = L->c[3 * i] - u[0], dy = L->c[3 * i + 1] - u[1], dz = L->c[3 * i + 2] - u[2];
            double v = f[i];
            for (int e = 0; e < a; ++e) v *= dx;
            for (int e = 0; e < b; ++e) v *= dy;
            for (int e = 0; e < c; ++e) v *= dz;
            m += v;
        }
        mu[k] = m / *rho;
        C[k] = m; /* orders 0 and 1: kappa itself */
    }
    for (int k = 0; k < 27; ++k) {
        if (cum_order(k) < 2) continue;
        double kk = 0.0;
        for (int t = 0; t < g_cum.nterm[k]; ++t) {
            double v = g_cum.coef[k][t];
            for (int b = 0; b < g_cum.nblk[k][t]; ++b) v *= mu[g_cum.blk[k][t][b]];
            kk += v;
        }
        C[k] = *rho * kk;
    }
}

#define CI(a, b, c) ((a) + 3 * (b) + 9 * (c))

static void cumulant_relax(const orc_params *p, double rho, double *C)
{
    const double w1 = p->omega;
    const double *s = p->cum_s; /* groups 2..10 */
    /* [1] shear, [2] bulk */
    double dxy = C[CI(2, 0, 0)] - C[CI(0, 2, 0)], dxz = C[CI(2, 0, 0)] - C[CI(0, 0, 2)];
    double tr = C[CI(2, 0, 0)] + C[CI(0, 2, 0)] + C[CI(0, 0, 2)];
    dxy -= w1 * dxy;
    dxz -= w1 * dxz;
    tr -= s[0] * (tr - rho);
    C[CI(2, 0, 0)] = (dxy + dxz + tr) / 3.0;
    C[CI(0, 2, 0)] = C[CI(2, 0, 0)] - dxy;
    C[CI(0, 0, 2)] = C[CI(2, 0, 0)] - dxz;
    C[CI(1, 1, 0)] -= w1 * C[CI(1, 1, 0)];
    C[CI(1, 0, 1)] -= w1 * C[CI(1, 0, 1)];
    C[CI(0, 1, 1)] -= w1 * C[CI(0, 1, 1)];
    /* [3], [4] third order in pairs, [5] C_111 */
    const int pr[3][2] = {{CI(1, 2, 0), CI(1, 0, 2)}, {CI(2, 1, 0), CI(0, 1, 2)}, {CI(2, 0, 1), CI(0, 2, 1)}};
    for (int k = 0; k < 3; ++k) {
        double sm = C[pr[k][0]] + C[pr[k][1]], df = C[pr[k][0]] - C[pr[k][1]];
        sm -= s[1] * sm;
        df -= s[2] * df;
        C[pr[k][0]] = 0.5 * (sm + df);
        C[pr[k][1]] = 0.5 * (sm - df);
    }
    C[CI(1, 1, 1)] -= s[3] * C[CI(1, 1, 1)];
    /* [6], [7] the diagonal-pair fourth-order cumulants, [8] the mixed ones */
    {
        double a = C[CI(2, 2, 0)], b = C[CI(2, 0, 2)], c = C[CI(0, 2, 2)];
        double d1 = a - 2.0 * b + c, d2 = a + b - 2.0 * c, t = a + b + c;
        d1 -= s[4] * d1;
        d2 -= s[4] * d2;
        t -= s[5] * t;
        C[CI(2, 2, 0)] = (d1 + d2 + t) / 3.0;
        C[CI(2, 0, 2)] = (t - d1) / 3.0;
        C[CI(0, 2, 2)] = (t - d2) / 3.0;
    }
    C[CI(2, 1, 1)] -= s[6] * C[CI(2, 1, 1)];
    C[CI(1, 2, 1)] -= s[6] * C[CI(1, 2, 1)];
    C[CI(1, 1, 2)] -= s[6] * C[CI(1, 1, 2)];
    /* [9] fifth, [10] sixth order */
    C[CI(2, 2, 1)] -= s[7] * C[CI(2, 2, 1)];
    C[CI(2, 1, 2)] -= s[7] * C[CI(2, 1, 2)];
    C[CI(1, 2, 2)] -= s[7] * C[CI(1, 2, 2)];
    C[CI(2, 2, 2)] -= s[8] * C[CI(2, 2, 2)];
}

/* populations from rho, u and the density-scaled cumulants (orders 0 and 1: kappa itself) */
static void cumulants_to_f(const lattice_t *L, double rho, const double u[3], const double *C, double *f)
{
    double mu[27];
    int ord[27];
    for (int k = 0; k < 27; ++k) ord[k] = cum_order(k);
    for (int k = 0; k < 27; ++k)
        if (ord[k] < 2) mu[k] = C[k] / rho;
    for (int o = 2; o <= 6; ++o)
        for (int k = 0; k < 27; ++k) {
            if (ord[k] != o) continue;
            double v = C[k] / rho; /* k_abc; the one-block term is mu_abc itself */
            for (int t = 0; t < g_cum.nterm[k]; ++t) {
                if (g_cum.nblk[k][t] == 1) continue;
                double w = g_cum.coef[k][t];
                for (int b = 0; b < g_cum.nblk[k][t]; ++b) w *= mu[g_cum.blk[k][t][b]];
                v -= w;
            }
            mu[k] = v;
        }
    /* kappa -> f, one axis at a time: g[a][b][c] indexes (x, y, z) slots, each either a
     * moment order or a velocity component (0, 1, 2 = -1, 0, +1) */
    double g[27];
    for (int k = 0; k < 27; ++k) g[k] = rho * mu[k];
    for (int ax = 0; ax < 3; ++ax) {
        const int stride = ax == 0 ? 1 : (ax == 1 ? 3 : 9);
        for (int k = 0; k < 27; ++k) {
            if ((k / stride) % 3 != 0) continue;
            double m0 = g[k], m1 = g[k + stride], m2 = g[k + 2 * stride], ua = u[ax];
            double A = m1 + ua * m0, B = m2 + 2.0 * ua * m1 + ua * ua * m0;
            g[k] = 0.5 * (B - A);           /* c = -1 */
            g[k + stride] = m0 - B;         /* c = 0 */
            g[k + 2 * stride] = 0.5 * (B + A); /* c = +1 */
        }
    }
    for (int i = 0; i < 27; ++i) {
        int k = (L->c[3 * i] + 1) + 3 * (L->c[3 * i + 1] + 1) + 9 * (L->c[3 * i + 2] + 1);
        f[i] = g[k];
    }
}

static void collide_cumulant(const lattice_t *L, const orc_params *p, const double *f, double *fout)
{
    double rho, u[3], C[27];
    cumulants(L, f, p->force, &rho, u, C);
    cumulant_relax(p, rho, C);
    C[CI(1, 0, 0)] = 0.5 * p->force[0];
    C[CI(0, 1, 0)] = 0.5 * p->force[1];
    C[CI(0, 0, 1)] = 0.5 * p->force[2];
    cumulants_to_f(L, rho, u, C, fout);
}

/* the density-scaled cumulants of one D3Q27 cell (see above; C[0] = rho, first order: the
 * central first moments) and its rho, u */
int orc_cumulants(const orc_params *p, const double *f, double *C, double *rho_u)
{
    lattice_t L;
    if (p->q != 27 || get_lattice(27, &L) != 0) return -1;
    double rho, u[3];
    cumulants(&L, f, p->force, &rho, u, C);
    if (rho_u) {
        rho_u[0] = rho;
        rho_u[1] = u[0];
        rho_u[2] = u[1];
        rho_u[3] = u[2];
    }
    return 0;
}

/* populations of one D3Q27 cell with density rho, velocity u and density-scaled cumulants C
 * (orders 0 and 1 are the central moments kappa_000 and kappa_100, kappa_010, kappa_001) */
int orc_cumulants_to_f(double rho, const double *u, const double *C, double *f)
{
    lattice_t L;
    if (get_lattice(27, &L) != 0) return -1;
    cumulants_to_f(&L, rho, u, C, f);
    return 0;
}

void orc_collide(const orc_params *p, const double *f, double *fout)
{
    lattice_t L;
    if (get_lattice(p->q, &L) != 0) return;
    if (p->collision == ORC_CUMULANT && L.q != 27) return;
    collide(&L, p, NULL, f, fout);
}

/* One cell under a closure: its omega+ and post-collision populations. */
double orc_collide_closure(const orc_params *p, const orc_closure *cl, const double *f, double *fout)
{
    lattice_t L;
    if (get_lattice(p->q, &L) != 0) return -1.0;
    double rho, u[3];
    moments_pre(&L, f, p->force, &rho, u);
    if (fout) collide(&L, p, cl, f, fout);
    return closure_omega(&L, p, cl, f, rho, u);
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------------------
 * Initial state.  Reading: the pre-collision populations at t = 0 are the equilibrium at
 * rho0 and u0 - F/(2 rho0), so that the half-force-corrected velocity of Eq. 1 equals the
 * requested u0; the stored state is their post-collision image f*(x, 0).
 * rho, u: N and 3N (SoA: u[a*N + cell]) arrays, cell = x + nx (y + ny z).
 * Non-fluid cells get all-zero PDFs.
 * ------------------------------------------------------------------------------------- */
int orc_init(const orc_params *p, const uint8_t *flags, const double *rho, const double *u, double *f)
{
    lattice_t L;
    if (get_lattice(p->q, &L) != 0) return -1;
    if (p->collision == ORC_CUMULANT && L.q != 27) return -5;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    const int q = L.q;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        if (flags[n] != ORC_FLUID) {
            for (int i = 0; i < q; ++i) f[i * N + n] = 0.0;
            continue;
        }
        double r = rho[n];
        double uu[3];
        for (int a = 0; a < 3; ++a) uu[a] = u[a * N + n] - 0.5 * p->force[a] / r;
        double feq[QMAX], fs[QMAX];
        equilibrium(&L, r, uu, feq);
        collide(&L, p, NULL, feq, fs);
        for (int i = 0; i < q; ++i) f[i * N + n] = fs[i];
    }
    return 0;
}

/* Kind of the cell at (x, y, z), which may lie outside the domain by one cell.
 * Periodic axes wrap.  A coordinate outside a non-periodic axis takes the kind of that
 * face; when it is outside on several non-periodic axes, the first of x, y, z decides
 * (reading: the paper does not treat domain corners).  *cell receives the wrapped linear
 * index for in-domain cells, *face the face index (2*axis+side) for outside cells. */
static int resolve(const orc_params *p, const uint8_t *flags, int x, int y, int z, int64_t *cell, int *face)
{
    int xyz[3] = {x, y, z};
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a) {
        if (xyz[a] >= 0 && xyz[a] < n[a]) continue;
        if (p->periodic[a]) {
            xyz[a] = (xyz[a] + n[a]) % n[a];
        }
    }
    for (int a = 0; a < 3; ++a) {
        if (xyz[a] < 0 || xyz[a] >= n[a]) {
            *face = 2 * a + (xyz[a] < 0 ? 0 : 1);
            return p->face_kind[*face];
        }
    }
    *cell = (int64_t)xyz[0] + (int64_t)n[0] * ((int64_t)xyz[1] + (int64_t)n[1] * xyz[2]);
    *face = -1;
    return flags[*cell];
}

/* ---------------------------------------------------------------------------------------
 * Time stepping in the push form of Eq. 2.
 *   f   : in/out, post-collision state f*(t) -> f*(t + nsteps)
 *   work: scratch array of the same size (pre-collision field of the next step)
 *   cell_u (3N, SoA) / cell_rho (N): wall velocity / density of interior VELOCITY and
 *   PRESSURE cells; may be NULL when the flag field has no such cells.
 * For each fluid x and direction i, with y = x + c_i:
 *   y fluid    : f_i(y, t+1)    = f*_i(x)
 *   y no-slip  : f_opp(x, t+1)  = f*_i(x)                                   (bounce-back)
 *   y velocity : f_opp(x, t+1)  = f*_i(x) - 6 w_i rho_w (c_i . u_w)       (moving wall)
 *   y pressure : f_opp(x, t+1)  = -f*_i(x) + 2 w_i rho_w [1 + 9/2 (c_i.u_b)^2 - 3/2 u_b^2]
 *                with u_b the velocity of x at time t (anti-bounce-back, no extrapolation)
 * The wall lies halfway between x and y.  Then every fluid cell collides.
 * ------------------------------------------------------------------------------------- */
int orc_run_closure(const orc_params *p, const orc_closure *cl, const uint8_t *flags, const double *cell_u,
                    const double *cell_rho, double *f, double *work, int64_t nsteps);
static int stream_pass(const lattice_t *Lp, const orc_params *p, const uint8_t *flags, const double *cell_u,
                       const double *cell_rho, const double *f, double *work);
static void zouhe_pass(const lattice_t *Lp, const orc_params *p, const uint8_t *flags, double *work);

int orc_run(const orc_params *p, const uint8_t *flags, const double *cell_u, const double *cell_rho, double *f,
            double *work, int64_t nsteps)
{
    return orc_run_closure(p, NULL, flags, cell_u, cell_rho, f, work, nsteps);
}

/* Time stepping as orc_run, with a locally varying omega+ from the closure. */
int orc_run_closure(const orc_params *p, const orc_closure *cl, const uint8_t *flags, const double *cell_u,
                    const double *cell_rho, double *f, double *work, int64_t nsteps)
{
    lattice_t L;
    if (get_lattice(p->q, &L) != 0) return -1;
    if (p->collision == ORC_CUMULANT && (L.q != 27 || (cl && cl->kind != 0))) return -5;
    const int q = L.q;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int a = 0; a < 6; ++a) {
        if (p->periodic[a / 2]) continue;
        int k = p->face_kind[a];
        if (k != ORC_NOSLIP && k != ORC_VELOCITY && k != ORC_PRESSURE && k != ORC_ZOUHE_VELOCITY &&
            k != ORC_ZOUHE_PRESSURE)
            return -2;
        if ((k == ORC_ZOUHE_VELOCITY || k == ORC_ZOUHE_PRESSURE) && L.q != 19) return -4;
    }

    for (int64_t step = 0; step < nsteps; ++step) {
        if (stream_pass(&L, p, flags, cell_u, cell_rho, f, work) != 0) return -3;
        zouhe_pass(&L, p, flags, work);
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < N; ++n) {
            if (flags[n] != ORC_FLUID) continue;
            double fin[QMAX], fout[QMAX];
            for (int i = 0; i < q; ++i) fin[i] = work[i * N + n];
            collide(&L, p, cl, fin, fout);
            for (int i = 0; i < q; ++i) f[i * N + n] = fout[i];
        }
    }
    return 0;
}

/* The streaming half of a step alone: the pre-collision field f(t + 1) of the post-collision
 * state f*(t), boundaries included (the first pass of orc_run); non-fluid cells get zeros. */
int orc_stream(const orc_params *p, const uint8_t *flags, const double *cell_u, const double *cell_rho,
               const double *f, double *fpre)
{
    lattice_t L;
    if (get_lattice(p->q, &L) != 0) return -1;
    for (int a = 0; a < 6; ++a) {
        if (p->periodic[a / 2]) continue;
        int k = p->face_kind[a];
        if (k != ORC_NOSLIP && k != ORC_VELOCITY && k != ORC_PRESSURE && k != ORC_ZOUHE_VELOCITY &&
            k != ORC_ZOUHE_PRESSURE)
            return -2;
        if ((k == ORC_ZOUHE_VELOCITY || k == ORC_ZOUHE_PRESSURE) && L.q != 19) return -4;
    }
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int i = 0; i < L.q; ++i)
        for (int64_t n = 0; n < N; ++n)
            if (flags[n] != ORC_FLUID) fpre[i * N + n] = 0.0;
    if (stream_pass(&L, p, flags, cell_u, cell_rho, f, fpre) != 0) return -3;
    zouhe_pass(&L, p, flags, fpre);
    return 0;
}

/* Push every post-collision PDF of f to its target (see above) into work. */
static int stream_pass(const lattice_t *Lp, const orc_params *p, const uint8_t *flags, const double *cell_u,
                       const double *cell_rho, const double *f, double *work)
{
    const lattice_t L = *Lp;
    const int nx = p->nx, ny = p->ny, nz = p->nz, q = L.q;
    const int64_t N = (int64_t)nx * ny * nz;
    int bad = 0;
    {
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int z = 0; z < nz; ++z) {
            for (int y = 0; y < ny; ++y) {
                for (int x = 0; x < nx; ++x) {
                    int64_t n = (int64_t)x + (int64_t)nx * ((int64_t)y + (int64_t)ny * z);
                    if (flags[n] != ORC_FLUID) continue;
                    double fs[QMAX];
                    for (int i = 0; i < q; ++i) fs[i] = f[i * N + n];
                    double rb = 0.0, ub[3] = {0.0, 0.0, 0.0};
                    int have_ub = 0;
                    for (int i = 0; i < q; ++i) {
                        int64_t m;
                        int face;
                        int kind = resolve(p, flags, x + L.c[3 * i], y + L.c[3 * i + 1], z + L.c[3 * i + 2], &m, &face);
                        int o = L.opp[i];
                        if (kind == ORC_FLUID) {
                            work[i * N + m] = fs[i];
                        } else if (kind == ORC_ZOUHE_VELOCITY || kind == ORC_ZOUHE_PRESSURE) {
                            /* leaves the domain through a wet-node face: nothing comes back here;
                               the node's incoming populations are reconstructed by zouhe_pass */
                        } else if (kind == ORC_NOSLIP) {
                            work[o * N + n] = fs[i];
                        } else if (kind == ORC_VELOCITY) {
                            double uw[3], rw;
                            if (face >= 0) {
                                for (int a = 0; a < 3; ++a) uw[a] = p->face_u[face][a];
                                rw = p->face_rho[face];
                            } else {
                                for (int a = 0; a < 3; ++a) uw[a] = cell_u[a * N + m];
                                rw = cell_rho[m];
                            }
                            double cu = L.c[3 * i] * uw[0] + L.c[3 * i + 1] * uw[1] + L.c[3 * i + 2] * uw[2];
                            work[o * N + n] = fs[i] - 6.0 * L.w[i] * rw * cu;
                        } else if (kind == ORC_PRESSURE) {
                            double rw = face >= 0 ? p->face_rho[face] : cell_rho[m];
                            if (!have_ub) {
                                moments_post(&L, fs, p->force, &rb, ub);
                                have_ub = 1;
                            }
                            double cu = L.c[3 * i] * ub[0] + L.c[3 * i + 1] * ub[1] + L.c[3 * i + 2] * ub[2];
                            double usq = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
                            work[o * N + n] = -fs[i] + 2.0 * L.w[i] * rw * (1.0 + 4.5 * cu * cu - 1.5 * usq);
                        } else {
                            bad = 1;
                        }
                    }
                    (void)rb;
                }
            }
        }
    }
    return bad ? -3 : 0;
}

/* ---------------------------------------------------------------------------------------
 * Wet-node velocity and pressure faces (Zou & He 1997; the paper cites the family of in- and
 * outflow conditions in Sec. 5.1.1), D3Q19.  The boundary node is the fluid cell of the first
 * layer at the face; after streaming, the populations entering it through the face (c_i.n > 0,
 * n the inward normal) are unknown.  With K0 = sum of the populations with c.n = 0 and Km = sum of
 * those with c.n < 0 (both known), mass and normal momentum give rho = K0 + 2 Km + j.n, where the
 * node's momentum is j = rho u - F/2 (the Guo half-force shift of Eq. 1).
 *   velocity face (u_w given):  rho = (K0 + 2 Km - F.n / 2) / (1 - u_w.n),  j = rho u_w - F/2;
 *   pressure face (rho_w given): rho = rho_w, tangential velocity zero,
 *                                j.n = rho_w - K0 - 2 Km,  j.t = -F.t / 2.
 * The unknowns take the known opposite population plus the equilibrium difference, with the
 * tangential momentum corrected (Hecht & Harting 2010 for D3Q19):
 *   c = n:          f_c = f_-c + j.n / 3
 *   c = n + s t:    f_c = f_-c + (j.n + s j.t) / 6 - s N_t,
 *                   N_t = (1/2) sum_{c_k.n = 0} (c_k.t) f_k - j.t / 3,
 * for the two tangential axes t and s = +-1.  Then the node collides as every fluid cell.
 * Reading: the wall sits at the node; the face's two tangential axes are periodic or the
 * node's neighbours along them are fluid (edges where two non-periodic faces meet are not
 * treated).  Populations entering the node from solid cells of the flag field are bounced back
 * by stream_pass before this pass.
 * ------------------------------------------------------------------------------------- */
static void zouhe_pass(const lattice_t *Lp, const orc_params *p, const uint8_t *flags, double *work)
{
    const lattice_t L = *Lp;
    const int n3[3] = {p->nx, p->ny, p->nz};
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
    for (int face = 0; face < 6; ++face) {
        const int kind = p->face_kind[face];
        const int a = face / 2, side = face % 2;
        if (p->periodic[a] || (kind != ORC_ZOUHE_VELOCITY && kind != ORC_ZOUHE_PRESSURE)) continue;
        const int nrm = side == 0 ? 1 : -1; /* inward normal along axis a */
        const int t1 = (a + 1) % 3, t2 = (a + 2) % 3;
        const int lay = side == 0 ? 0 : n3[a] - 1;
        const int e1 = n3[t1], e2 = n3[t2];
#pragma omp parallel for schedule(static)
        for (int v = 0; v < e2; ++v) {
            for (int w = 0; w < e1; ++w) {
                int xyz[3];
                xyz[a] = lay;
                xyz[t1] = w;
                xyz[t2] = v;
                const int64_t cell = (int64_t)xyz[0] + (int64_t)p->nx * ((int64_t)xyz[1] + (int64_t)p->ny * xyz[2]);
                if (flags[cell] != ORC_FLUID) continue;
                double K0 = 0.0, Km = 0.0, T[3] = {0.0, 0.0, 0.0};
                for (int i = 0; i < L.q; ++i) {
                    const int cn = L.c[3 * i + a] * nrm;
                    const double fi = work[i * N + cell];
                    if (cn == 0) {
                        K0 += fi;
                        for (int b = 0; b < 3; ++b) T[b] += L.c[3 * i + b] * fi;
                    } else if (cn < 0) {
                        Km += fi;
                    }
                }
                const double *F = p->force;
                double rho, j[3];
                if (kind == ORC_ZOUHE_VELOCITY) {
                    const double *uw = p->face_u[face];
                    rho = (K0 + 2.0 * Km - 0.5 * F[a] * nrm) / (1.0 - uw[a] * nrm);
                    for (int b = 0; b < 3; ++b) j[b] = rho * uw[b] - 0.5 * F[b];
                } else {
                    rho = p->face_rho[face];
                    for (int b = 0; b < 3; ++b) j[b] = -0.5 * F[b];
                    j[a] = (rho - K0 - 2.0 * Km) * nrm;
                }
                const double jn = j[a] * nrm;
                for (int i = 0; i < L.q; ++i) {
                    if (L.c[3 * i + a] * nrm <= 0) continue;
                    const int o = L.opp[i];
                    double fi = work[o * N + cell] + jn / 3.0;
                    const int tt = L.c[3 * i + t1] != 0 ? t1 : (L.c[3 * i + t2] != 0 ? t2 : -1);
                    if (tt >= 0) {
                        const double s = L.c[3 * i + tt];
                        const double Nt = 0.5 * T[tt] - j[tt] / 3.0;
                        fi = work[o * N + cell] + (jn + s * j[tt]) / 6.0 - s * Nt;
                    }
                    work[i * N + cell] = fi;
                }
            }
        }
    }
}

/* Output moments of the stored state (Eq. 1, with the Guo shift for a post-collision
 * state): rho = sum f*, u = (sum c f* - F/2) / rho.  Non-fluid cells give rho = u = 0. */
int orc_macroscopic(const orc_params *p, const uint8_t *flags, const double *f, double *rho, double *u)
{
    lattice_t L;
    if (get_lattice(p->q, &L) != 0) return -1;
    const int64_t N = (int64_t)p->nx * p->ny * p->nz;
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < N; ++n) {
        if (flags[n] != ORC_FLUID) {
            rho[n] = 0.0;
            u[n] = u[N + n] = u[2 * N + n] = 0.0;
            continue;
        }
        double fs[QMAX], r, uu[3];
        for (int i = 0; i < L.q; ++i) fs[i] = f[i * N + n];
        moments_post(&L, fs, p->force, &r, uu);
        rho[n] = r;
        for (int a = 0; a < 3; ++a) u[a * N + n] = uu[a];
    }
    return 0;
}

/* ---------------------------------------------------------------------------------------
 * Static 2:1 grid refinement, mass-conserving (Sec. 5.1.1: non-uniform grids by the method of
 * Rohde et al. 2006, which the paper names without giving its rules).  Reading, in the
 * volumetric form of that method:
 *   * cells are volumes and the populations densities in them; a coarse cell holds 2 x 2 x 2
 *     fine cells; the fine grid takes two steps per coarse step; its rates follow from the
 *     same physical viscosity under acoustic scaling, tau_f - 1/2 = 2 (tau_c - 1/2) (TRT: the
 *     same Lambda on both grids), and its body force is F_c / 2 (so that the force per volume
 *     and coarse step is the same);
 *   * geometry: the coarse grid covers the periodic nx x ny x nz box; the coarse columns
 *     x in [a, b) (periodic in x; 0 <= a < b <= nx, b - a < nx) are refined: the fine grid
 *     covers them with 2 (b - a) x 2 ny x 2 nz cells; y and z are periodic on both grids;
 *   * one coarse step:
 *     1. explosion: a layer of fine ghost cells two deep on each side of the fine grid
 *        (inside the coarse columns a - 1 and b) takes the post-collision populations of the
 *        coarse cell it lies in, the same value in each of its 8 fine cells (no
 *        interpolation, no rescaling of the non-equilibrium part);
 *     2. two fine steps, each: push-stream every fine cell, ghosts included (values that would
 *        leave the ghost layer are dropped), then collide the fine cells (ghosts keep what
 *        streamed into them);
 *     3. coalescence and coarse streaming: push-stream the coarse cells; a coarse population
 *        whose target lies in the refined columns is dropped (the explosion delivered it); a
 *        coarse cell next to the refined columns takes, for each direction whose source lies
 *        there, the mean of that direction's values over the 8 fine ghost cells inside it
 *        (the fine populations that left the fine grid into its volume during the two fine
 *        steps); then collide the coarse cells.
 *   Each population that crosses the interface is counted once on each side, so the mass
 *   sum_coarse f + (1/8) sum_fine f is conserved exactly in exact arithmetic, and so is the
 *   momentum apart from the body force.
 * State: fc[i][z][y][x] over the coarse box (the refined columns hold zeros),
 * ff[i][zf][yf][xf] over the fine grid, both post-collision.
 * ------------------------------------------------------------------------------------- */
int orc_refine_fine_params(const orc_params *pc, int32_t a, int32_t b, orc_params *pf)
{
    if (pc->collision != ORC_SRT && pc->collision != ORC_TRT) return -1;
    if (!(pc->periodic[0] && pc->periodic[1] && pc->periodic[2])) return -2;
    if (a < 0 || b > pc->nx || a >= b || b - a >= pc->nx) return -3;
    if (!(pc->omega > 0.0 && pc->omega < 2.0)) return -4;
    *pf = *pc;
    pf->nx = 2 * (b - a);
    pf->ny = 2 * pc->ny;
    pf->nz = 2 * pc->nz;
    pf->omega = 1.0 / (0.5 + 2.0 * (1.0 / pc->omega - 0.5));
    for (int k = 0; k < 3; ++k) pf->force[k] = 0.5 * pc->force[k];
    return 0;
}

int orc_refine_run(const orc_params *pc, int32_t a, int32_t b, double *fc, double *ff, int64_t nsteps)
{
    lattice_t L;
    orc_params pf;
    int r = orc_refine_fine_params(pc, a, b, &pf);
    if (r != 0) return r;
    if (get_lattice(pc->q, &L) != 0) return -1;
    const int q = L.q;
    const int nx = pc->nx, ny = pc->ny, nz = pc->nz;
    const int64_t Nc = (int64_t)nx * ny * nz;
    const int nf = pf.nx, nyf = pf.ny, nzf = pf.nz;
    const int nxg = nf + 4; /* fine grid with its two ghost columns on each side: xg = xf + 2 */
    const int64_t Ng = (int64_t)nxg * nyf * nzf;
    const int64_t Nf = (int64_t)nf * nyf * nzf;
    double *g = calloc((size_t)q * Ng, sizeof(double));
    double *gw = calloc((size_t)q * Ng, sizeof(double));
    double *cw = calloc((size_t)q * Nc, sizeof(double));
    if (!g || !gw || !cw) {
        free(g);
        free(gw);
        free(cw);
        return -6;
    }
#define IN_SLAB(x) (((x) - a + nx) % nx < b - a)
    for (int i = 0; i < q; ++i)
        for (int z = 0; z < nzf; ++z)
            for (int y = 0; y < nyf; ++y)
                for (int x = 0; x < nf; ++x)
                    g[i * Ng + ((int64_t)z * nyf + y) * nxg + x + 2] = ff[i * Nf + ((int64_t)z * nyf + y) * nf + x];
    const int left = (a - 1 + nx) % nx, right = b % nx; /* coarse columns holding the ghosts */
    for (int64_t step = 0; step < nsteps; ++step) {
        /* 1. explosion */
        for (int i = 0; i < q; ++i)
            for (int z = 0; z < nzf; ++z)
                for (int y = 0; y < nyf; ++y)
                    for (int s = 0; s < 4; ++s) {
                        const int xg = s < 2 ? s : nf + s; /* 0, 1 | nf + 2, nf + 3 */
                        const int xc = s < 2 ? left : right;
                        g[i * Ng + ((int64_t)z * nyf + y) * nxg + xg] = fc[i * Nc + ((int64_t)(z / 2) * ny + y / 2) * nx + xc];
                    }
        /* 2. two fine steps */
        for (int sub = 0; sub < 2; ++sub) {
            memset(gw, 0, sizeof(double) * (size_t)q * Ng);
            for (int z = 0; z < nzf; ++z)
                for (int y = 0; y < nyf; ++y)
                    for (int x = 0; x < nxg; ++x)
                        for (int i = 0; i < q; ++i) {
                            const int xt = x + L.c[3 * i];
                            if (xt < 0 || xt >= nxg) continue;
                            const int yt = (y + L.c[3 * i + 1] + nyf) % nyf, zt = (z + L.c[3 * i + 2] + nzf) % nzf;
                            gw[i * Ng + ((int64_t)zt * nyf + yt) * nxg + xt] = g[i * Ng + ((int64_t)z * nyf + y) * nxg + x];
                        }
            memcpy(g, gw, sizeof(double) * (size_t)q * Ng);
#pragma omp parallel for schedule(static)
            for (int64_t n = 0; n < Ng; ++n) {
                const int xg = (int)(n % nxg);
                if (xg < 2 || xg >= nf + 2) continue; /* ghosts are not collided */
                double fin[QMAX], fout[QMAX];
                for (int i = 0; i < q; ++i) fin[i] = g[i * Ng + n];
                collide(&L, &pf, NULL, fin, fout);
                for (int i = 0; i < q; ++i) g[i * Ng + n] = fout[i];
            }
        }
        /* 3. coarse streaming with coalescence, then the coarse collision */
        memset(cw, 0, sizeof(double) * (size_t)q * Nc);
        for (int z = 0; z < nz; ++z)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    if (IN_SLAB(x)) continue;
                    for (int i = 0; i < q; ++i) {
                        const int xt = (x + L.c[3 * i] + nx) % nx;
                        if (IN_SLAB(xt)) continue;
                        const int yt = (y + L.c[3 * i + 1] + ny) % ny, zt = (z + L.c[3 * i + 2] + nz) % nz;
                        cw[i * Nc + ((int64_t)zt * ny + yt) * nx + xt] = fc[i * Nc + ((int64_t)z * ny + y) * nx + x];
                    }
                }
        for (int side = 0; side < 2; ++side) {
            const int xc = side == 0 ? left : right;
            const int xg0 = side == 0 ? 0 : nf + 2;
            for (int z = 0; z < nz; ++z)
                for (int y = 0; y < ny; ++y)
                    for (int i = 0; i < q; ++i) {
                        const int xs = (xc - L.c[3 * i] + nx) % nx;
                        if (!IN_SLAB(xs)) continue;
                        double s = 0.0;
                        for (int dz = 0; dz < 2; ++dz)
                            for (int dy = 0; dy < 2; ++dy)
                                for (int dx = 0; dx < 2; ++dx)
                                    s += g[i * Ng + ((int64_t)(2 * z + dz) * nyf + 2 * y + dy) * nxg + xg0 + dx];
                        cw[i * Nc + ((int64_t)z * ny + y) * nx + xc] = s / 8.0;
                    }
        }
#pragma omp parallel for schedule(static)
        for (int64_t n = 0; n < Nc; ++n) {
            if (IN_SLAB((int)(n % nx))) continue;
            double fin[QMAX], fout[QMAX];
            for (int i = 0; i < q; ++i) fin[i] = cw[i * Nc + n];
            collide(&L, pc, NULL, fin, fout);
            for (int i = 0; i < q; ++i) fc[i * Nc + n] = fout[i];
        }
    }
#undef IN_SLAB
    for (int i = 0; i < q; ++i)
        for (int z = 0; z < nzf; ++z)
            for (int y = 0; y < nyf; ++y)
                for (int x = 0; x < nf; ++x)
                    ff[i * Nf + ((int64_t)z * nyf + y) * nf + x] = g[i * Ng + ((int64_t)z * nyf + y) * nxg + x + 2];
    free(g);
    free(gw);
    free(cw);
    return 0;
}
