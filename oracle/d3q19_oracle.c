/*
 * d3q19_oracle.c -- FP64 CPU oracle of the coupled MRT / AMRT lattice
 * Boltzmann method on D3Q19 (see d3q19_oracle.h for the readings).
 *
 * TEST INFRASTRUCTURE ONLY (tests, the smoke check and the benchmark's CPU
 * baseline).  Plain loops, one node at a time, in the order of the paper's
 * equations; no blocking or fusion.
 */
#include "d3q19_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define CS2 (1.0 / 3.0)

/* D3Q19 velocities and weights in the order of the lattice remark of Sec. 3.1 */
static const int E[Q][3] = {{0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},  {0, -1, 0}, {0, 0, 1},  {0, 0, -1},
                            {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {-1, 0, 1},
                            {1, 0, -1}, {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};

typedef struct {
    double w[Q];
    double M[Q][Q];    /* M[k][i]: moment k of direction i */
    double Minv[Q][Q]; /* M^-1 = M^T diag(1 / |row_k|^2) (orthogonal rows) */
} lat3_t;

static void lat_init(lat3_t* L) {
    for (int i = 0; i < Q; ++i) {
        const int n2 = E[i][0] * E[i][0] + E[i][1] * E[i][1] + E[i][2] * E[i][2];
        L->w[i] = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        const double ex = E[i][0], ey = E[i][1], ez = E[i][2], e2 = n2;
        const double row[Q] = {1.0,
                               19.0 * e2 - 30.0,
                               (21.0 * e2 * e2 - 53.0 * e2 + 24.0) / 2.0,
                               ex,
                               (5.0 * e2 - 9.0) * ex,
                               ey,
                               (5.0 * e2 - 9.0) * ey,
                               ez,
                               (5.0 * e2 - 9.0) * ez,
                               3.0 * ex * ex - e2,
                               (3.0 * e2 - 5.0) * (3.0 * ex * ex - e2),
                               ey * ey - ez * ez,
                               (3.0 * e2 - 5.0) * (ey * ey - ez * ez),
                               ex * ey,
                               ey * ez,
                               ex * ez,
                               (ey * ey - ez * ez) * ex,
                               (ez * ez - ex * ex) * ey,
                               (ex * ex - ey * ey) * ez};
        for (int k = 0; k < Q; ++k) L->M[k][i] = row[k];
    }
    for (int k = 0; k < Q; ++k) {
        double n = 0.0;
        for (int i = 0; i < Q; ++i) n += L->M[k][i] * L->M[k][i];
        for (int i = 0; i < Q; ++i) L->Minv[i][k] = L->M[k][i] / n;
    }
}

int od3_lattice(int* e, double* w, double* M) {
    lat3_t L;
    lat_init(&L);
    for (int i = 0; i < Q; ++i) {
        for (int c = 0; c < 3; ++c) e[3 * i + c] = E[i][c];
        w[i] = L.w[i];
        for (int k = 0; k < Q; ++k) M[k * Q + i] = L.M[k][i];
    }
    return 0;
}

int od3_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* 3x3 inverse (symmetric input) */
static int inv3(const double A[3][3], double B[3][3]) {
    const double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1], c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2],
                 c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
    const double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
    if (!(fabs(det) > 0.0)) return -1;
    B[0][0] = c00 / det;
    B[1][0] = c01 / det;
    B[2][0] = c02 / det;
    B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
    B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
    B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
    B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
    B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
    B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
    return 0;
}

/* K = (D / (d Cs^2 tau) + I/2)^-1 (the D -> K map of Sec. 3.1, PC12-14) */
static void K_from_D(const double* D6, double d, double tau, double K[3][3]) {
    const double sc = 1.0 / (d * CS2 * tau);
    const double A[3][3] = {{D6[0] * sc + 0.5, D6[1] * sc, D6[2] * sc},
                            {D6[1] * sc, D6[3] * sc + 0.5, D6[4] * sc},
                            {D6[2] * sc, D6[4] * sc, D6[5] * sc + 0.5}};
    inv3(A, K);
}

/* phi^eq_i = w_i [Theta + (a Theta).e_i / Cs^2 + (C + (d - 1) Cs^2 Theta I) : U_i / (2 Cs^4)],
 * U_i = e_i e_i - Cs^2 I, C = (a a) Theta */
static void feq3(const lat3_t* L, double Theta, const double a[3], double d, double* out) {
    for (int i = 0; i < Q; ++i) {
        double BU = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                const double U = E[i][r] * E[i][c] - (r == c ? CS2 : 0.0);
                const double B = a[r] * a[c] * Theta + (r == c ? (d - 1.0) * CS2 * Theta : 0.0);
                BU += B * U;
            }
        const double aT = (a[0] * E[i][0] + a[1] * E[i][1] + a[2] * E[i][2]) * Theta;
        out[i] = L->w[i] * (Theta + aT / CS2 + BU / (2.0 * CS2 * CS2));
    }
}

/* aleph_j = d phi^eq_j / d Theta / w_j (the adjoint equilibrium weights) */
static void aleph3(const double a[3], double d, double* out) {
    for (int j = 0; j < Q; ++j) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c)
                s += (a[r] * a[c] + (r == c ? (d - 1.0) * CS2 : 0.0)) * (E[j][r] * E[j][c] - (r == c ? CS2 : 0.0));
        out[j] = 1.0 + (a[0] * E[j][0] + a[1] * E[j][1] + a[2] * E[j][2]) / CS2 + s / (2.0 * CS2 * CS2);
    }
}

typedef struct {
    double Ku[3][3], Kv[3][3];
    double a[3];
    double aleph_u[Q], aleph_v[Q];
    double wt_v[Q]; /* w~_i = w_i (1 + V.e_i / Cs^2), V = (I - K_v/2) a */
} node3d_t;

static void node_params(const lat3_t* L, const od3_problem* p, size_t k, node3d_t* nd) {
    K_from_D(p->Du + 6 * k, p->d_u, p->tau, nd->Ku);
    K_from_D(p->Dv + 6 * k, p->d_v, p->tau, nd->Kv);
    for (int c = 0; c < 3; ++c) nd->a[c] = p->a ? p->a[3 * k + c] : 0.0;
    aleph3(nd->a, p->d_u, nd->aleph_u);
    aleph3(nd->a, p->d_v, nd->aleph_v);
    double V[3];
    for (int r = 0; r < 3; ++r) {
        V[r] = nd->a[r];
        for (int c = 0; c < 3; ++c) V[r] -= 0.5 * nd->Kv[r][c] * nd->a[c];
    }
    for (int i = 0; i < Q; ++i)
        nd->wt_v[i] = L->w[i] * (1.0 + (V[0] * E[i][0] + V[1] * E[i][1] + V[2] * E[i][2]) / CS2);
}

/* relaxation matrix: free rates on the non-flux moments, K on (j_x, j_y, j_z) */
static const int RATE[Q] = {0, 1, 2, -1, 3, -1, 3, -1, 3, 4, 5, 4, 5, 4, 4, 4, 6, 6, 6};
static const int JIDX[3] = {3, 5, 7};

static void Pi3(const double s[7], const double K[3][3], double Pi[Q][Q]) {
    memset(Pi, 0, sizeof(double) * Q * Q);
    for (int k = 0; k < Q; ++k)
        if (RATE[k] >= 0) Pi[k][k] = s[RATE[k]];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Pi[JIDX[r]][JIDX[c]] = K[r][c];
}

/* P = f - M^-1 Pi (M f - M f^eq) */
static void collide(const lat3_t* L, const double Pi[Q][Q], const double* f, const double* feq, double* out) {
    double dm[Q], r[Q];
    for (int k = 0; k < Q; ++k) {
        dm[k] = 0.0;
        for (int i = 0; i < Q; ++i) dm[k] += L->M[k][i] * (f[i] - feq[i]);
    }
    for (int k = 0; k < Q; ++k) {
        r[k] = 0.0;
        for (int l = 0; l < Q; ++l) r[k] += Pi[k][l] * dm[l];
    }
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += L->Minv[i][k] * r[k];
        out[i] = f[i] - s;
    }
}

/* (M^-1 Pi M)^T rho */
static void collide_T(const lat3_t* L, const double Pi[Q][Q], const double* rho, double* mt) {
    double y[Q], z[Q];
    for (int k = 0; k < Q; ++k) {
        y[k] = 0.0;
        for (int i = 0; i < Q; ++i) y[k] += L->Minv[i][k] * rho[i];
    }
    for (int l = 0; l < Q; ++l) {
        z[l] = 0.0;
        for (int k = 0; k < Q; ++k) z[l] += Pi[k][l] * y[k];
    }
    for (int j = 0; j < Q; ++j) {
        mt[j] = 0.0;
        for (int l = 0; l < Q; ++l) mt[j] += L->M[l][j] * z[l];
    }
}

static double c_now(const od3_problem* p, int n) { return (p->source_order == 1 || n == 0) ? p->tau : 1.5 * p->tau; }
static double c_prev(const od3_problem* p, int n) { return (p->source_order == 1 || n == 0) ? 0.0 : -0.5 * p->tau; }

/* grad v from v's first non-equilibrium moment (relation C146, kappa_x = 0):
 * G = -(K_v (j_v - a v)/tau + K_v a Phi_v / 2) / (d_v Cs^2) */
static void grad_v(const od3_problem* p, const node3d_t* nd, double Tv, const double jv[3], double Phi,
                   double G[3]) {
    double r[3];
    for (int c = 0; c < 3; ++c) r[c] = (jv[c] - nd->a[c] * Tv) / p->tau;
    for (int c = 0; c < 3; ++c) {
        double s = 0.0;
        for (int l = 0; l < 3; ++l) s += nd->Kv[c][l] * (r[l] + 0.5 * nd->a[l] * Phi);
        G[c] = -s / (p->d_v * CS2);
    }
}

typedef struct {
    double Tu, Tv, Phi, G[3];
} st3d_t;

/* one collision at a node: f[2][Q] -> P[2][Q] */
static void collide_node(const lat3_t* L, const od3_problem* p, const node3d_t* nd, int n, const double* f, double g,
                         double Phi_prev, double* P, st3d_t* st) {
    double Tu = 0.0, Tv = 0.0, jv[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        Tu += f[i];
        Tv += f[Q + i];
        for (int c = 0; c < 3; ++c) jv[c] += E[i][c] * f[Q + i];
    }
    const double Phi = p->r_vu * Tu + p->r_vv * Tv + g;
    const double Pp = (n == 0) ? Phi : Phi_prev;
    double G[3];
    grad_v(p, nd, Tv, jv, Phi, G);
    double Pi[Q][Q], feq[Q];
    Pi3(p->s, nd->Ku, Pi);
    feq3(L, Tu, nd->a, p->d_u, feq);
    collide(L, Pi, f, feq, P);
    Pi3(p->s, nd->Kv, Pi);
    feq3(L, Tv, nd->a, p->d_v, feq);
    collide(L, Pi, f + Q, feq, P + Q);
    for (int i = 0; i < Q; ++i) {
        double src = p->tau * nd->wt_v[i] * Phi;
        if (p->source_order != 1) src += 0.5 * p->tau * nd->wt_v[i] * (Phi - Pp);
        P[Q + i] += src;
    }
    /* tau S_u,i = (w_i / Cs^2) e_i . (K_u chi u G) */
    double KF[3];
    for (int r = 0; r < 3; ++r) {
        KF[r] = 0.0;
        for (int c = 0; c < 3; ++c) KF[r] += nd->Ku[r][c] * p->chi * Tu * G[c];
    }
    for (int i = 0; i < Q; ++i) P[i] += L->w[i] / CS2 * (E[i][0] * KF[0] + E[i][1] * KF[1] + E[i][2] * KF[2]);
    if (st) {
        st->Tu = Tu;
        st->Tv = Tv;
        st->Phi = Phi;
        for (int c = 0; c < 3; ++c) st->G[c] = G[c];
    }
}

static inline size_t nidx(const od3_problem* p, int x, int y, int z) {
    return ((size_t)z * p->ny + y) * p->nx + x;
}

/* periodic streaming: pull f_i(x) = P_i(x - e_i) (forward), or
 * rho_i(x) = psi_i(x + e_i) (adjoint) */
static void stream(const od3_problem* p, const double* P, double* f, int adjoint) {
    const int nx = p->nx, ny = p->ny, nz = p->nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < Q; ++i) {
                        const int sg = adjoint ? 1 : -1;
                        const int xs = (x + sg * E[i][0] + nx) % nx, ys = (y + sg * E[i][1] + ny) % ny,
                                  zs = (z + sg * E[i][2] + nz) % nz;
                        f[(nidx(p, x, y, z) * 2 + s) * Q + i] = P[(nidx(p, xs, ys, zs) * 2 + s) * Q + i];
                    }
}

static int run_forward(const od3_problem* p, const double* g, double* fN, double* traj, double* Phi_traj,
                       double* mass_u, double* mass_v, double* sum_phi) {
    lat3_t L;
    lat_init(&L);
    const size_t nn = (size_t)p->nx * p->ny * p->nz, npop = nn * 2 * Q;
    double* f = calloc(npop, sizeof(double));
    double* P = calloc(npop, sizeof(double));
    double* Phi = calloc(nn, sizeof(double));
    double* Tn = calloc(nn * 2, sizeof(double));
    node3d_t* nodes = malloc(sizeof(node3d_t) * nn);
    if (!f || !P || !Phi || !Tn || !nodes) return -2;
    for (size_t k = 0; k < nn; ++k) {
        node_params(&L, p, k, &nodes[k]);
        feq3(&L, p->u0[k], nodes[k].a, p->d_u, f + k * 2 * Q);
        feq3(&L, p->v0[k], nodes[k].a, p->d_v, f + k * 2 * Q + Q);
    }
    for (int n = 0; n < p->N; ++n) {
        if (traj) memcpy(traj + (size_t)n * npop, f, sizeof(double) * npop);
#pragma omp parallel for schedule(static)
        for (long long kk = 0; kk < (long long)nn; ++kk) {
            const size_t k = (size_t)kk;
            st3d_t st;
            const double gv = g ? g[(size_t)n * nn + k] : 0.0;
            collide_node(&L, p, &nodes[k], n, f + k * 2 * Q, gv, Phi[k], P + k * 2 * Q, &st);
            Phi[k] = st.Phi;
            Tn[2 * k] = st.Tu;
            Tn[2 * k + 1] = st.Tv;
        }
        if (Phi_traj) memcpy(Phi_traj + (size_t)n * nn, Phi, sizeof(double) * nn);
        if (mass_u || mass_v || sum_phi) {
            double mu = 0.0, mv = 0.0, sp = 0.0;
            for (size_t k = 0; k < nn; ++k) {
                mu += Tn[2 * k];
                mv += Tn[2 * k + 1];
                sp += Phi[k];
            }
            if (mass_u) mass_u[n] = mu;
            if (mass_v) mass_v[n] = mv;
            if (sum_phi) sum_phi[n] = sp;
        }
        stream(p, P, f, 0);
    }
    memcpy(fN, f, sizeof(double) * npop);
    free(f);
    free(P);
    free(Phi);
    free(Tn);
    free(nodes);
    return 0;
}

static double cost(const od3_problem* p, const double* fN, const double* g, double* uN, double* vN, double* wu) {
    const size_t nn = (size_t)p->nx * p->ny * p->nz;
    double s = 0.0, pen = 0.0;
    for (size_t k = 0; k < nn; ++k) {
        double Tu = 0.0, Tv = 0.0;
        for (int i = 0; i < Q; ++i) {
            Tu += fN[k * 2 * Q + i];
            Tv += fN[k * 2 * Q + Q + i];
        }
        if (uN) uN[k] = Tu;
        if (vN) vN[k] = Tv;
        const double d = Tu - p->u_tgt[k];
        if (wu) wu[k] = d;
        s += 0.5 * d * d;
    }
    if (g)
        for (size_t q = 0; q < (size_t)p->N * nn; ++q) pen += g[q] * g[q];
    return s + p->alpha * pen;
}

int od3_forward(const od3_problem* p, const double* g, double* J, double* uN, double* vN) {
    const size_t nn = (size_t)p->nx * p->ny * p->nz;
    double* fN = malloc(sizeof(double) * nn * 2 * Q);
    if (!fN) return -2;
    const int rc = run_forward(p, g, fN, NULL, NULL, NULL, NULL, NULL);
    if (rc) return rc;
    const double c = cost(p, fN, g, uN, vN, NULL);
    if (J) *J = c;
    free(fN);
    return 0;
}

int od3_forward_trace(const od3_problem* p, const double* g, double* mass_u, double* mass_v, double* sum_phi) {
    const size_t nn = (size_t)p->nx * p->ny * p->nz;
    double* fN = malloc(sizeof(double) * nn * 2 * Q);
    if (!fN) return -2;
    const int rc = run_forward(p, g, fN, NULL, NULL, mass_u, mass_v, sum_phi);
    free(fN);
    return rc;
}

int od3_tlm(const od3_problem* p, const double* g, const double* dg, const double* df0, double* duN, double* dvN) {
    lat3_t L;
    lat_init(&L);
    const size_t nn = (size_t)p->nx * p->ny * p->nz, npop = nn * 2 * Q;
    double *f = calloc(npop, sizeof(double)), *P = calloc(npop, sizeof(double));
    double *df = calloc(npop, sizeof(double)), *dP = calloc(npop, sizeof(double));
    double *Phi = calloc(nn, sizeof(double)), *dPhi = calloc(nn, sizeof(double));
    node3d_t* nodes = malloc(sizeof(node3d_t) * nn);
    if (!f || !P || !df || !dP || !Phi || !dPhi || !nodes) return -2;
    for (size_t k = 0; k < nn; ++k) {
        node_params(&L, p, k, &nodes[k]);
        feq3(&L, p->u0[k], nodes[k].a, p->d_u, f + k * 2 * Q);
        feq3(&L, p->v0[k], nodes[k].a, p->d_v, f + k * 2 * Q + Q);
    }
    if (df0) memcpy(df, df0, sizeof(double) * npop);
    for (int n = 0; n < p->N; ++n) {
#pragma omp parallel for schedule(static)
        for (long long kk = 0; kk < (long long)nn; ++kk) {
            const size_t k = (size_t)kk;
            const node3d_t* nd = &nodes[k];
            st3d_t st;
            const double gv = g ? g[(size_t)n * nn + k] : 0.0, dgv = dg ? dg[(size_t)n * nn + k] : 0.0;
            collide_node(&L, p, nd, n, f + k * 2 * Q, gv, Phi[k], P + k * 2 * Q, &st);
            /* tangent of the local map (linear in f except through u G) */
            const double* dfk = df + k * 2 * Q;
            double* dPk = dP + k * 2 * Q;
            double dTu = 0.0, dTv = 0.0, djv[3] = {0, 0, 0};
            for (int i = 0; i < Q; ++i) {
                dTu += dfk[i];
                dTv += dfk[Q + i];
                for (int c = 0; c < 3; ++c) djv[c] += E[i][c] * dfk[Q + i];
            }
            const double dPh = p->r_vu * dTu + p->r_vv * dTv + dgv;
            const double dPp = (n == 0) ? dPh : dPhi[k];
            double dG[3];
            grad_v(p, nd, dTv, djv, dPh, dG);
            double Pi[Q][Q], dfeq[Q];
            Pi3(p->s, nd->Ku, Pi);
            feq3(&L, dTu, nd->a, p->d_u, dfeq);
            collide(&L, Pi, dfk, dfeq, dPk);
            Pi3(p->s, nd->Kv, Pi);
            feq3(&L, dTv, nd->a, p->d_v, dfeq);
            collide(&L, Pi, dfk + Q, dfeq, dPk + Q);
            for (int i = 0; i < Q; ++i) {
                double src = p->tau * nd->wt_v[i] * dPh;
                if (p->source_order != 1) src += 0.5 * p->tau * nd->wt_v[i] * (dPh - dPp);
                dPk[Q + i] += src;
            }
            double dKF[3];
            for (int r = 0; r < 3; ++r) {
                dKF[r] = 0.0;
                for (int c = 0; c < 3; ++c) dKF[r] += nd->Ku[r][c] * p->chi * (dTu * st.G[c] + st.Tu * dG[c]);
            }
            for (int i = 0; i < Q; ++i)
                dPk[i] += L.w[i] / CS2 * (E[i][0] * dKF[0] + E[i][1] * dKF[1] + E[i][2] * dKF[2]);
            Phi[k] = st.Phi;
            dPhi[k] = dPh;
        }
        stream(p, P, f, 0);
        stream(p, dP, df, 0);
    }
    for (size_t k = 0; k < nn; ++k) {
        double du = 0.0, dv = 0.0;
        for (int i = 0; i < Q; ++i) {
            du += df[k * 2 * Q + i];
            dv += df[k * 2 * Q + Q + i];
        }
        if (duN) duN[k] = du;
        if (dvN) dvN[k] = dv;
    }
    free(f);
    free(P);
    free(df);
    free(dP);
    free(Phi);
    free(dPhi);
    free(nodes);
    return 0;
}

/* One node of the AMRT step at step n, the exact transpose of collide_node:
 * from the pulled adjoint populations rho [2][Q] and the node's forward state
 * at step n (pre-collision f [2][Q], Phi = Phi^n), the node's adjoint
 * populations psi [2][Q], sigma^n and the adjoint of Phi^n (its use at step n
 * and, when has_next, with c'_{n+1} sigma^{n+1} at step n + 1). */
static void adjoint_local(const lat3_t* L, const od3_problem* p, const node3d_t* nd, int n, const double* fk,
                          double Phi, const double* rk, int has_next, double sig_next, double* psi_out,
                          double* sig_out, double* aPhi_out) {
    const double sc = 1.0 / (p->d_v * CS2);
    double Tu = 0.0, Tv = 0.0, jv[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i) {
        Tu += fk[i];
        Tv += fk[Q + i];
        for (int cc = 0; cc < 3; ++cc) jv[cc] += E[i][cc] * fk[Q + i];
    }
    double G[3];
    grad_v(p, nd, Tv, jv, Phi, G);
    /* transposed collisions with the adjoint-equilibrium broadcast */
    double out[2 * Q], Pi[Q][Q], mt[Q];
    for (int s = 0; s < 2; ++s) {
        Pi3(p->s, s == 0 ? nd->Ku : nd->Kv, Pi);
        collide_T(L, Pi, rk + s * Q, mt);
        const double* al = s == 0 ? nd->aleph_u : nd->aleph_v;
        double Tcal = 0.0;
        for (int i = 0; i < Q; ++i) Tcal += L->w[i] * al[i] * mt[i];
        for (int i = 0; i < Q; ++i) out[s * Q + i] = rk[s * Q + i] - mt[i] + Tcal;
    }
    /* adjoint of tau S_u = (w_i / Cs^2) e_i . K_u F, F = chi u G */
    double Y[3] = {0, 0, 0};
    for (int i = 0; i < Q; ++i)
        for (int cc = 0; cc < 3; ++cc) Y[cc] += rk[i] * L->w[i] / CS2 * E[i][cc];
    double aF[3];
    for (int cc = 0; cc < 3; ++cc) {
        aF[cc] = 0.0;
        for (int r = 0; r < 3; ++r) aF[cc] += nd->Ku[r][cc] * Y[r];
    }
    double aTu = 0.0, aTv = 0.0, aPhi = 0.0, aG[3], aj[3];
    for (int cc = 0; cc < 3; ++cc) {
        aTu += p->chi * G[cc] * aF[cc];
        aG[cc] = p->chi * Tu * aF[cc];
    }
    /* G = -(K_v (j_v - a v)/tau + K_v a Phi/2) / (d_v Cs^2) */
    double KtG[3];
    for (int cc = 0; cc < 3; ++cc) {
        KtG[cc] = 0.0;
        for (int r = 0; r < 3; ++r) KtG[cc] += nd->Kv[r][cc] * aG[r];
    }
    double aKG = 0.0;
    for (int cc = 0; cc < 3; ++cc) {
        aj[cc] = -KtG[cc] * sc / p->tau;
        aKG += nd->a[cc] * KtG[cc];
    }
    aTv += aKG * sc / p->tau;
    aPhi += -0.5 * aKG * sc;
    /* the source w~ (c_n Phi^n + c'_n Phi^{n-1}) and the use of Phi^n at step n+1 */
    double sig = 0.0;
    for (int i = 0; i < Q; ++i) sig += rk[Q + i] * nd->wt_v[i];
    aPhi += c_now(p, n) * sig;
    if (has_next) aPhi += c_prev(p, n + 1) * sig_next;
    *sig_out = sig;
    aTu += p->r_vu * aPhi;
    aTv += p->r_vv * aPhi;
    *aPhi_out = aPhi;
    for (int i = 0; i < Q; ++i) {
        psi_out[i] = out[i] + aTu;
        psi_out[Q + i] = out[Q + i] + aTv + E[i][0] * aj[0] + E[i][1] * aj[1] + E[i][2] * aj[2];
    }
}

int od3_adjoint(const od3_problem* p, const double* g, const double* seed_u, const double* seed_v, double* dJdg,
                double* psi0, double* J) {
    lat3_t L;
    lat_init(&L);
    const int N = p->N;
    const size_t nn = (size_t)p->nx * p->ny * p->nz, npop = nn * 2 * Q;
    double* traj = malloc(sizeof(double) * npop * (size_t)N);
    double* Phi_traj = malloc(sizeof(double) * nn * (size_t)N);
    double* fN = malloc(sizeof(double) * npop);
    double* psi = calloc(npop, sizeof(double));
    double* rho = calloc(npop, sizeof(double));
    double* sig_next = calloc(nn, sizeof(double));
    double* sig_now = calloc(nn, sizeof(double));
    double* wu = malloc(sizeof(double) * nn);
    node3d_t* nodes = malloc(sizeof(node3d_t) * nn);
    if (!traj || !Phi_traj || !fN || !psi || !rho || !sig_next || !sig_now || !wu || !nodes) return -2;
    const int rc = run_forward(p, g, fN, traj, Phi_traj, NULL, NULL, NULL);
    if (rc) return rc;
    for (size_t k = 0; k < nn; ++k) node_params(&L, p, k, &nodes[k]);
    const double c = cost(p, fN, g, NULL, NULL, wu);
    if (J) *J = c;
    /* final condition: psi_Theta,i(T) = d I0 / d f_Theta,i (a broadcast per species) */
    for (size_t k = 0; k < nn; ++k)
        for (int i = 0; i < Q; ++i) {
            psi[k * 2 * Q + i] = seed_u ? seed_u[k] : wu[k];
            psi[k * 2 * Q + Q + i] = seed_v ? seed_v[k] : 0.0;
        }
    for (int n = N - 1; n >= 0; --n) {
        stream(p, psi, rho, 1); /* along -e_i, backward in time */
        const double* f = traj + (size_t)n * npop;
#pragma omp parallel for schedule(static)
        for (long long kk = 0; kk < (long long)nn; ++kk) {
            const size_t k = (size_t)kk;
            double aPhi;
            adjoint_local(&L, p, &nodes[k], n, f + k * 2 * Q, Phi_traj[(size_t)n * nn + k], rho + k * 2 * Q,
                          n + 1 <= N - 1, sig_next[k], psi + k * 2 * Q, &sig_now[k], &aPhi);
            if (dJdg) {
                const double gv = g ? g[(size_t)n * nn + k] : 0.0;
                dJdg[(size_t)n * nn + k] = aPhi + 2.0 * p->alpha * gv;
            }
        }
        double* t = sig_next;
        sig_next = sig_now;
        sig_now = t;
    }
    if (psi0) memcpy(psi0, psi, sizeof(double) * npop);
    free(traj);
    free(Phi_traj);
    free(fN);
    free(psi);
    free(rho);
    free(sig_next);
    free(sig_now);
    free(wu);
    free(nodes);
    return 0;
}

int od3_collide_node(const od3_problem* p, int x, int y, int z, int n, const double* f, double g,
                     double Phi_prev, double* P, double* Phi_out) {
    lat3_t L;
    lat_init(&L);
    if (x < 0 || y < 0 || z < 0 || x >= p->nx || y >= p->ny || z >= p->nz) return -3;
    node3d_t nd;
    node_params(&L, p, nidx(p, x, y, z), &nd);
    st3d_t st;
    collide_node(&L, p, &nd, n, f, g, Phi_prev, P, &st);
    *Phi_out = st.Phi;
    return 0;
}

int od3_adjoint_node(const od3_problem* p, int x, int y, int z, int n, const double* f, double g,
                     const double* rho, int has_next, double sigma_next, double* psi, double* sigma_out,
                     double* lam_Phi) {
    lat3_t L;
    lat_init(&L);
    if (x < 0 || y < 0 || z < 0 || x >= p->nx || y >= p->ny || z >= p->nz) return -3;
    node3d_t nd;
    node_params(&L, p, nidx(p, x, y, z), &nd);
    double Tu = 0.0, Tv = 0.0;
    for (int i = 0; i < Q; ++i) {
        Tu += f[i];
        Tv += f[Q + i];
    }
    const double Phi = p->r_vu * Tu + p->r_vv * Tv + g; /* as collide_node forms Phi^n */
    adjoint_local(&L, p, &nd, n, f, Phi, rho, has_next, sigma_next, psi, sigma_out, lam_Phi);
    return 0;
}
