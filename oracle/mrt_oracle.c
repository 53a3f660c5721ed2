/*
 * mrt_oracle.c -- FP64 CPU oracle (test infrastructure; see mrt_oracle.h).
 *
 * Plain, slow and written to be checked against the paper by eye: one node at
 * a time, explicit moment matrices, explicit 2x2 inverses.  Where the paper is
 * silent the readings are:
 *   - h = tau = c = 1 is allowed but tau is kept symbolic; C_s^2 = c^2/3 (Sec. 3.1).
 *   - D2Q5 (not in the paper): the first five D2Q9 velocities, w0 = 1/3,
 *     w1..4 = 1/6, moments (rho, j_x, j_y, e, p_xx).
 *   - kappa_t = 1, kappa_x = 0 in (LBE); the tau^2/2 dPhi/dt term is the
 *     explicit characteristic difference of the remark after (UGS):
 *     (tau/2)(Phi^n - Phi^{n-1}); Phi^{-1} := Phi^0.
 *   - grad v in S_u is taken locally from v's first non-equilibrium moment,
 *     solving the first-order relation (C146) for grad v:
 *       G = -( K_v (j_v - a v)/tau + (1/2) K_v a Phi_v ) / (d_v C_s^2).
 *   - f^0 = phi^eq(Theta_0) (no streaming before the first collision).
 *   - halfway bounce-back at solid nodes: f_i(x) = P_{opp(i)}(x) when x - e_i
 *     is solid.
 *   - control g^n drives step n -> n+1 (n = 0..N-1); J = 1/2 sum (u^N - u_tgt)^2
 *     + alpha sum_{n<N} sum g^2; the gradient is the exact gradient of this J.
 *
 * The per-node loops (collision, streaming, set-up) run rows in parallel with
 * OpenMP when it is compiled in; every node's arithmetic and every sum's order
 * are those of the serial loops, so results are bitwise the same for any
 * thread count (or_set_threads).
 */
#include "mrt_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)

typedef struct {
    int Q;
    int e[9][2];
    double w[9];
    double M[9][9];
    double Minv[9][9];
    int opp[9];
} lattice_t;

/* Gauss-Jordan inverse of a Q x Q matrix with partial pivoting. */
static int invert(int Q, const double A[9][9], double X[9][9]) {
    double W[9][18];
    for (int i = 0; i < Q; ++i) {
        for (int j = 0; j < Q; ++j) {
            W[i][j] = A[i][j];
            W[i][Q + j] = (i == j) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < Q; ++c) {
        int piv = c;
        for (int r = c + 1; r < Q; ++r)
            if (fabs(W[r][c]) > fabs(W[piv][c])) piv = r;
        if (fabs(W[piv][c]) < 1e-14) return -1;
        if (piv != c)
            for (int j = 0; j < 2 * Q; ++j) {
                double t = W[c][j];
                W[c][j] = W[piv][j];
                W[piv][j] = t;
            }
        double d = W[c][c];
        for (int j = 0; j < 2 * Q; ++j) W[c][j] /= d;
        for (int r = 0; r < Q; ++r) {
            if (r == c) continue;
            double f = W[r][c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * Q; ++j) W[r][j] -= f * W[c][j];
        }
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j) X[i][j] = W[i][Q + j];
    return 0;
}

/* D2Q9 velocities, weights and the Gram-Schmidt moment matrix M0 as printed
 * in Sec. 3.1 (E0 = I because c = 1).  D2Q5: first five D2Q9 velocities. */
static int lattice_init(lattice_t* L, int Q) {
    static const int e9[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                 {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    static const double M9[9][9] = {
        {1, 1, 1, 1, 1, 1, 1, 1, 1},
        {-4, -1, -1, -1, -1, 2, 2, 2, 2},
        {4, -2, -2, -2, -2, 1, 1, 1, 1},
        {0, 1, 0, -1, 0, 1, -1, -1, 1},
        {0, -2, 0, 2, 0, 1, -1, -1, 1},
        {0, 0, 1, 0, -1, 1, 1, -1, -1},
        {0, 0, -2, 0, 2, 1, 1, -1, -1},
        {0, 1, -1, 1, -1, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 1, -1, 1, -1}};
    static const double M5[5][5] = {
        {1, 1, 1, 1, 1},
        {0, 1, 0, -1, 0},
        {0, 0, 1, 0, -1},
        {-4, 1, 1, 1, 1},
        {0, 1, -1, 1, -1}};
    memset(L, 0, sizeof(*L));
    if (Q != 9 && Q != 5) return -1;
    L->Q = Q;
    for (int i = 0; i < Q; ++i) {
        L->e[i][0] = e9[i][0];
        L->e[i][1] = e9[i][1];
    }
    if (Q == 9) {
        L->w[0] = 4.0 / 9.0;
        for (int i = 1; i <= 4; ++i) L->w[i] = 1.0 / 9.0;
        for (int i = 5; i <= 8; ++i) L->w[i] = 1.0 / 36.0;
        for (int i = 0; i < 9; ++i)
            for (int j = 0; j < 9; ++j) L->M[i][j] = M9[i][j];
    } else {
        L->w[0] = 1.0 / 3.0;
        for (int i = 1; i <= 4; ++i) L->w[i] = 1.0 / 6.0;
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) L->M[i][j] = M5[i][j];
    }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            if (L->e[j][0] == -L->e[i][0] && L->e[j][1] == -L->e[i][1]) L->opp[i] = j;
    return invert(Q, (const double(*)[9])L->M, L->Minv);
}

/* ---------------------------------------------------------------- node data */

typedef struct {
    double Ku[2][2], Kv[2][2]; /* relaxation blocks K_Theta (Sec. 3.1, Pi) */
    double a[2];               /* convection velocity */
    double aleph_u[9], aleph_v[9]; /* d phi^eq_j / d Theta = w_j aleph_j */
    double wt_v[9];            /* w~_i = w_i (1 + V.e_i / C_s^2)   (PhiS) */
} node_t;

static void inv2(const double A[2][2], double X[2][2]) {
    double det = A[0][0] * A[1][1] - A[0][1] * A[1][0];
    X[0][0] = A[1][1] / det;
    X[0][1] = -A[0][1] / det;
    X[1][0] = -A[1][0] / det;
    X[1][1] = A[0][0] / det;
}

/* K from D_Theta = d_Theta C_s^2 tau (K^{-1} - I/2)   (choice after PC13). */
static void K_from_D(const double* D3, double d, double tau, double K[2][2]) {
    double Kinv[2][2];
    double sc = 1.0 / (d * CS2 * tau);
    Kinv[0][0] = D3[0] * sc + 0.5;
    Kinv[0][1] = D3[1] * sc;
    Kinv[1][0] = D3[1] * sc;
    Kinv[1][1] = D3[2] * sc + 0.5;
    inv2(Kinv, K);
}

/* Equilibrium (phieq) with T = a Theta and C = (a (x) a) Theta (tensorC):
 *   phi^eq_i = w_i [ Theta + (a Theta).e_i / Cs^2
 *                   + (C + d Cs^2 Theta I - Cs^2 Theta I) : U_i / (2 Cs^4) ],
 *   U_i = e_i (x) e_i - Cs^2 I. */
static void feq_lat(const lattice_t* L, double Theta, const double a[2], double d, double* out) {
    for (int i = 0; i < L->Q; ++i) {
        double ex = L->e[i][0], ey = L->e[i][1];
        double U[2][2] = {{ex * ex - CS2, ex * ey}, {ey * ex, ey * ey - CS2}};
        double C[2][2] = {{a[0] * a[0] * Theta, a[0] * a[1] * Theta},
                          {a[1] * a[0] * Theta, a[1] * a[1] * Theta}};
        double B[2][2];
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                B[r][c] = C[r][c] + ((r == c) ? (d * CS2 * Theta - CS2 * Theta) : 0.0);
        double BU = B[0][0] * U[0][0] + B[0][1] * U[0][1] + B[1][0] * U[1][0] + B[1][1] * U[1][1];
        out[i] = L->w[i] * (Theta + (a[0] * Theta * ex + a[1] * Theta * ey) / CS2 +
                            BU / (2.0 * CS2 * CS2));
    }
}

/* aleph_j of the adjoint equilibrium (the formula for d phi^eq_j / d phi_i):
 *   aleph_j = 1 + dT/dTheta . e_j / Cs^2 + (dC/dTheta + (d - 1) Cs^2 I) : U_j / (2 Cs^4). */
static void aleph_lat(const lattice_t* L, const double a[2], double d, double* out) {
    for (int j = 0; j < L->Q; ++j) {
        double ex = L->e[j][0], ey = L->e[j][1];
        double U[2][2] = {{ex * ex - CS2, ex * ey}, {ey * ex, ey * ey - CS2}};
        double dC[2][2] = {{a[0] * a[0], a[0] * a[1]}, {a[1] * a[0], a[1] * a[1]}};
        double s = 0.0;
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 2; ++c)
                s += (dC[r][c] + ((r == c) ? (d - 1.0) * CS2 : 0.0)) * U[r][c];
        out[j] = 1.0 + (a[0] * ex + a[1] * ey) / CS2 + s / (2.0 * CS2 * CS2);
    }
}

static void node_params(const lattice_t* L, const or_problem* p, int x, int y, node_t* nd) {
    int k = y * p->nx + x;
    K_from_D(p->Du + 3 * k, p->d_u, p->tau, nd->Ku);
    K_from_D(p->Dv + 3 * k, p->d_v, p->tau, nd->Kv);
    nd->a[0] = p->a ? p->a[2 * k] : 0.0;
    nd->a[1] = p->a ? p->a[2 * k + 1] : 0.0;
    aleph_lat(L, nd->a, p->d_u, nd->aleph_u);
    aleph_lat(L, nd->a, p->d_v, nd->aleph_v);
    /* V_v = (K^{-1} - (kappa_x/2) I)^{-1} (K^{-1} - I/2) dT/dTheta with kappa_x = 0 */
    double Kinv[2][2], A[2][2], Ainv[2][2], Bm[2][2], V[2];
    inv2(nd->Kv, Kinv);
    for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c) {
            A[r][c] = Kinv[r][c]; /* - (kappa_x/2) I with kappa_x = 0 */
            Bm[r][c] = Kinv[r][c] - ((r == c) ? 0.5 : 0.0);
        }
    inv2(A, Ainv);
    double Ba[2] = {Bm[0][0] * nd->a[0] + Bm[0][1] * nd->a[1], Bm[1][0] * nd->a[0] + Bm[1][1] * nd->a[1]};
    V[0] = Ainv[0][0] * Ba[0] + Ainv[0][1] * Ba[1];
    V[1] = Ainv[1][0] * Ba[0] + Ainv[1][1] * Ba[1];
    for (int i = 0; i < L->Q; ++i)
        nd->wt_v[i] = L->w[i] * (1.0 + (V[0] * L->e[i][0] + V[1] * L->e[i][1]) / CS2);
}

/* Relaxation matrix Pi_Theta in moment space (Sec. 3.1): block diagonal
 * diag(s0,s1,s2) + [[k11,0,k12],[0,s3,0],[k21,0,k22]] + diag(s4,s5,s6) on the
 * D2Q9 moment order (rho, e, eps, j_x, q_x, j_y, q_y, p_xx, p_xy).  D2Q5 moment
 * order (rho, j_x, j_y, e, p_xx): s0 + K + diag(s1, s5). */
static void Pi_matrix(const lattice_t* L, const or_problem* p, const double K[2][2], double Pi[9][9]) {
    memset(Pi, 0, sizeof(double) * 81);
    const double* s = p->s;
    if (L->Q == 9) {
        Pi[0][0] = s[0];
        Pi[1][1] = s[1];
        Pi[2][2] = s[2];
        Pi[3][3] = K[0][0];
        Pi[3][5] = K[0][1];
        Pi[4][4] = s[3];
        Pi[5][3] = K[1][0];
        Pi[5][5] = K[1][1];
        Pi[6][6] = s[4];
        Pi[7][7] = s[5];
        Pi[8][8] = s[6];
    } else {
        Pi[0][0] = s[0];
        Pi[1][1] = K[0][0];
        Pi[1][2] = K[0][1];
        Pi[2][1] = K[1][0];
        Pi[2][2] = K[1][1];
        Pi[3][3] = s[1];
        Pi[4][4] = s[5];
    }
}

/* MRT collision in moment space (MF), (MC):  m = M f,  m^eq = M f^eq,
 * m^col = m - Pi (m - m^eq),  returns  f - M^{-1} Pi (m - m^eq). */
static void mrt_collide(const lattice_t* L, const double Pi[9][9], const double* f, const double* feq,
                        double* out) {
    int Q = L->Q;
    double m[9], meq[9], dm[9];
    for (int k = 0; k < Q; ++k) {
        m[k] = 0.0;
        meq[k] = 0.0;
        for (int i = 0; i < Q; ++i) {
            m[k] += L->M[k][i] * f[i];
            meq[k] += L->M[k][i] * feq[i];
        }
    }
    for (int k = 0; k < Q; ++k) {
        dm[k] = 0.0;
        for (int l = 0; l < Q; ++l) dm[k] += Pi[k][l] * (m[l] - meq[l]);
    }
    for (int i = 0; i < Q; ++i) {
        double s = 0.0;
        for (int k = 0; k < Q; ++k) s += L->Minv[i][k] * dm[k];
        out[i] = f[i] - s;
    }
}

/* Transposed MRT collision operator applied to an adjoint vector:
 * m~ = Lambda^T rho with Lambda = M^{-1} Pi M, i.e. M^T Pi^T M^{-T} rho. */
static void mrt_collide_T(const lattice_t* L, const double Pi[9][9], const double* rho, double* mt) {
    int Q = L->Q;
    double y[9], z[9];
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

static int is_solid(const or_problem* p, int x, int y) {
    return p->solid ? p->solid[y * p->nx + x] != 0 : 0;
}

/* index of node x in the control vector, or -1 */
static int ctrl_index(const or_problem* p, int x, int y) {
    int cx = x - p->cx0, cy = y - p->cy0;
    if (cx < 0 || cy < 0 || cx >= p->cnx || cy >= p->cny) return -1;
    if (is_solid(p, x, y)) return -1;
    if (p->cmask && !p->cmask[cy * p->cnx + cx]) return -1;
    return cy * p->cnx + cx;
}

/* coefficient of Phi^n in the step-n source: tau at n = 0 (Phi^{-1} := Phi^0),
 * 3 tau / 2 afterwards; tau when the (tau/2) dPhi term is dropped. */
static double c_now(const or_problem* p, int n) {
    if (p->source_order == 1 || n == 0) return p->tau;
    return 1.5 * p->tau;
}
static double c_prev(const or_problem* p, int n) {
    if (p->source_order == 1 || n == 0) return 0.0;
    return -0.5 * p->tau;
}

/* ----------------------------------------------------- local forward step */

typedef struct {
    double Theta_u, Theta_v, jv[2], Phi, G[2];
} state_t;

/* grad v from the first non-equilibrium moment of v (reading of C146). */
static void grad_v(const or_problem* p, const node_t* nd, double Theta_v, const double jv[2], double Phi,
                   double G[2]) {
    double r[2];
    for (int c = 0; c < 2; ++c) r[c] = (jv[c] - nd->a[c] * Theta_v) / p->tau;
    double Kr[2] = {nd->Kv[0][0] * r[0] + nd->Kv[0][1] * r[1], nd->Kv[1][0] * r[0] + nd->Kv[1][1] * r[1]};
    double Ka[2] = {nd->Kv[0][0] * nd->a[0] + nd->Kv[0][1] * nd->a[1],
                    nd->Kv[1][0] * nd->a[0] + nd->Kv[1][1] * nd->a[1]};
    for (int c = 0; c < 2; ++c) G[c] = -(Kr[c] + 0.5 * Ka[c] * Phi) / (p->d_v * CS2);
}

static void collide_local(const lattice_t* L, const or_problem* p, const node_t* nd, int n, const double* f_u,
                          const double* f_v, double g, double Phi_prev, double* P_u, double* P_v,
                          state_t* st) {
    int Q = L->Q;
    double Tu = 0.0, Tv = 0.0, jv[2] = {0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        Tu += f_u[i];
        Tv += f_v[i];
        jv[0] += L->e[i][0] * f_v[i];
        jv[1] += L->e[i][1] * f_v[i];
    }
    double Phi = p->r_vu * Tu + p->r_vv * Tv + g;
    if (n == 0) Phi_prev = Phi;
    double G[2];
    grad_v(p, nd, Tv, jv, Phi, G);

    double Pi[9][9], feq[9];
    /* species u: MRT collision + tau S_u, S_u,i = w_i/Cs^2 e_i.(A_u grad v),
     * A_u = K_u D_{u,1} / tau with D_{u,1} = chi u I (S, choice after PC13) */
    Pi_matrix(L, p, nd->Ku, Pi);
    feq_lat(L, Tu, nd->a, p->d_u, feq);
    mrt_collide(L, Pi, f_u, feq, P_u);
    double AG[2];
    for (int c = 0; c < 2; ++c)
        AG[c] = (nd->Ku[c][0] * G[0] + nd->Ku[c][1] * G[1]) * p->chi * Tu / p->tau;
    for (int i = 0; i < Q; ++i)
        P_u[i] += p->tau * L->w[i] / CS2 * (L->e[i][0] * AG[0] + L->e[i][1] * AG[1]);
    /* species v: MRT collision + tau Phi_i + (tau/2)(Phi_i^n - Phi_i^{n-1}) */
    Pi_matrix(L, p, nd->Kv, Pi);
    feq_lat(L, Tv, nd->a, p->d_v, feq);
    mrt_collide(L, Pi, f_v, feq, P_v);
    for (int i = 0; i < Q; ++i) {
        double src = p->tau * nd->wt_v[i] * Phi;
        if (p->source_order != 1) src += 0.5 * p->tau * nd->wt_v[i] * (Phi - Phi_prev);
        P_v[i] += src;
    }
    if (st) {
        st->Theta_u = Tu;
        st->Theta_v = Tv;
        st->jv[0] = jv[0];
        st->jv[1] = jv[1];
        st->Phi = Phi;
        st->G[0] = G[0];
        st->G[1] = G[1];
    }
}

int or_collide_node(const or_problem* p, int x, int y, int n, const double* f_u, const double* f_v, double g,
                    double Phi_prev, double* P_u, double* P_v, double* Phi_out) {
    lattice_t L;
    if (lattice_init(&L, p->Q)) return -1;
    node_t nd;
    node_params(&L, p, x, y, &nd);
    state_t st;
    collide_local(&L, p, &nd, n, f_u, f_v, g, Phi_prev, P_u, P_v, &st);
    if (Phi_out) *Phi_out = st.Phi;
    return 0;
}

/* ---------------------------------------------------------- full forward */

/* pull streaming with halfway bounce-back: f_i(x) = P_i(x - e_i), or
 * P_opp(i)(x) when x - e_i is solid.  Arrays [ny][nx][2][Q]. */
static void stream_pull(const lattice_t* L, const or_problem* p, const double* P, double* f) {
    int Q = L->Q, nx = p->nx, ny = p->ny;
    memset(f, 0, sizeof(double) * (size_t)nx * ny * 2 * Q);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            for (int s = 0; s < 2; ++s)
                for (int i = 0; i < Q; ++i) {
                    int xs = (x - L->e[i][0] + nx) % nx, ys = (y - L->e[i][1] + ny) % ny;
                    double val;
                    if (is_solid(p, xs, ys))
                        val = P[((size_t)(y * nx + x) * 2 + s) * Q + L->opp[i]];
                    else
                        val = P[((size_t)(ys * nx + xs) * 2 + s) * Q + i];
                    f[((size_t)(y * nx + x) * 2 + s) * Q + i] = val;
                }
        }
}

/* adjoint of stream_pull: rho_j(y) = psi_j(y + e_j), or psi_opp(j)(y) when
 * y + e_j is solid -- streaming along -e_j backward in time (end of Sec. 3.2.1). */
static void stream_pull_T(const lattice_t* L, const or_problem* p, const double* psi, double* rho) {
    int Q = L->Q, nx = p->nx, ny = p->ny;
    memset(rho, 0, sizeof(double) * (size_t)nx * ny * 2 * Q);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            for (int s = 0; s < 2; ++s)
                for (int j = 0; j < Q; ++j) {
                    int xd = (x + L->e[j][0] + nx) % nx, yd = (y + L->e[j][1] + ny) % ny;
                    double val;
                    if (is_solid(p, xd, yd))
                        val = psi[((size_t)(y * nx + x) * 2 + s) * Q + L->opp[j]];
                    else
                        val = psi[((size_t)(yd * nx + xd) * 2 + s) * Q + j];
                    rho[((size_t)(y * nx + x) * 2 + s) * Q + j] = val;
                }
        }
}

static void init_populations(const lattice_t* L, const or_problem* p, double* f) {
    int Q = L->Q, nx = p->nx, ny = p->ny;
    memset(f, 0, sizeof(double) * (size_t)nx * ny * 2 * Q);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            int k = y * nx + x;
            double a[2] = {p->a ? p->a[2 * k] : 0.0, p->a ? p->a[2 * k + 1] : 0.0};
            feq_lat(L, p->u0[k], a, p->d_u, f + ((size_t)k * 2 + 0) * Q);
            feq_lat(L, p->v0[k], a, p->d_v, f + ((size_t)k * 2 + 1) * Q);
        }
}

static double g_at(const or_problem* p, const double* g, int n, int x, int y) {
    int c = ctrl_index(p, x, y);
    if (c < 0 || !g) return 0.0;
    return g[(size_t)n * p->cnx * p->cny + c];
}

/* One full forward run.  traj (optional): pre-collision populations f^n for
 * n = 0..N-1, [N][ny][nx][2][Q]; Phi_traj: Phi^n, [N][ny][nx]. */
static int run_forward(const or_problem* p, const double* g, double* fN, double* traj, double* Phi_traj,
                       double* mass_u, double* mass_v, double* sum_phi) {
    lattice_t L;
    if (lattice_init(&L, p->Q)) return -1;
    int Q = p->Q, nx = p->nx, ny = p->ny;
    size_t nn = (size_t)nx * ny, npop = nn * 2 * Q;
    double* f = calloc(npop, sizeof(double));
    double* P = calloc(npop, sizeof(double));
    double* Phi = calloc(nn, sizeof(double));
    node_t* nodes = malloc(sizeof(node_t) * nn);
    double* Th = (mass_u || mass_v || sum_phi) ? calloc(2 * nn, sizeof(double)) : NULL;
    if (!f || !P || !Phi || !nodes || ((mass_u || mass_v || sum_phi) && !Th)) return -2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) node_params(&L, p, x, y, &nodes[y * nx + x]);
    init_populations(&L, p, f);
    for (int n = 0; n < p->N; ++n) {
        if (traj) memcpy(traj + (size_t)n * npop, f, sizeof(double) * npop);
        memset(P, 0, sizeof(double) * npop);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (is_solid(p, x, y)) continue;
                size_t k = (size_t)y * nx + x;
                state_t st;
                collide_local(&L, p, &nodes[k], n, f + (k * 2) * Q, f + (k * 2 + 1) * Q, g_at(p, g, n, x, y),
                              Phi[k], P + (k * 2) * Q, P + (k * 2 + 1) * Q, &st);
                Phi[k] = st.Phi;
                if (Th) {
                    Th[2 * k] = st.Theta_u;
                    Th[2 * k + 1] = st.Theta_v;
                }
            }
        double mu = 0.0, mv = 0.0, sp = 0.0;
        if (Th)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    if (is_solid(p, x, y)) continue;
                    size_t k = (size_t)y * nx + x;
                    mu += Th[2 * k];
                    mv += Th[2 * k + 1];
                    sp += Phi[k];
                }
        if (Phi_traj) memcpy(Phi_traj + (size_t)n * nn, Phi, sizeof(double) * nn);
        if (mass_u) mass_u[n] = mu;
        if (mass_v) mass_v[n] = mv;
        if (sum_phi) sum_phi[n] = sp;
        stream_pull(&L, p, P, f);
    }
    memcpy(fN, f, sizeof(double) * npop);
    free(f);
    free(P);
    free(Phi);
    free(nodes);
    free(Th);
    return 0;
}

static double control_penalty(const or_problem* p, const double* g) {
    double s = 0.0;
    if (!g) return 0.0;
    for (int n = 0; n < p->N; ++n)
        for (int y = 0; y < p->ny; ++y)
            for (int x = 0; x < p->nx; ++x) {
                int c = ctrl_index(p, x, y);
                if (c < 0) continue;
                double v = g[(size_t)n * p->cnx * p->cny + c];
                s += v * v;
            }
    return p->alpha * s;
}

static void macro_fields(const or_problem* p, const double* f, double* u, double* v) {
    int Q = p->Q;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            size_t k = (size_t)y * p->nx + x;
            double su = 0.0, sv = 0.0;
            if (!is_solid(p, x, y))
                for (int i = 0; i < Q; ++i) {
                    su += f[(k * 2) * Q + i];
                    sv += f[(k * 2 + 1) * Q + i];
                }
            if (u) u[k] = su;
            if (v) v[k] = sv;
        }
}

static double terminal_cost(const or_problem* p, const double* u) {
    double s = 0.0;
    for (int y = 0; y < p->ny; ++y)
        for (int x = 0; x < p->nx; ++x) {
            if (is_solid(p, x, y)) continue;
            size_t k = (size_t)y * p->nx + x;
            double d = u[k] - p->u_tgt[k];
            s += 0.5 * d * d;
        }
    return s;
}

int or_forward(const or_problem* p, const double* g, double* J, double* uN, double* vN) {
    size_t nn = (size_t)p->nx * p->ny;
    double* fN = malloc(sizeof(double) * nn * 2 * p->Q);
    double* u = malloc(sizeof(double) * nn);
    if (!fN || !u) return -2;
    int rc = run_forward(p, g, fN, NULL, NULL, NULL, NULL, NULL);
    if (rc) return rc;
    macro_fields(p, fN, u, vN);
    if (uN) memcpy(uN, u, sizeof(double) * nn);
    if (J) *J = terminal_cost(p, u) + control_penalty(p, g);
    free(fN);
    free(u);
    return 0;
}

int or_forward_trace(const or_problem* p, const double* g, double* mass_u, double* mass_v, double* sum_phi) {
    size_t nn = (size_t)p->nx * p->ny;
    double* fN = malloc(sizeof(double) * nn * 2 * p->Q);
    if (!fN) return -2;
    int rc = run_forward(p, g, fN, NULL, NULL, mass_u, mass_v, sum_phi);
    free(fN);
    return rc;
}

/* ------------------------------------------------- tangent-linear model */

int or_tlm(const or_problem* p, const double* g, const double* dg, const double* df0, double* duN,
           double* dvN, double* dJ) {
    lattice_t L;
    if (lattice_init(&L, p->Q)) return -1;
    int Q = p->Q, nx = p->nx, ny = p->ny;
    size_t nn = (size_t)nx * ny, npop = nn * 2 * Q;
    double *f = calloc(npop, sizeof(double)), *P = calloc(npop, sizeof(double));
    double *df = calloc(npop, sizeof(double)), *dP = calloc(npop, sizeof(double));
    double *Phi = calloc(nn, sizeof(double)), *dPhi = calloc(nn, sizeof(double));
    node_t* nodes = malloc(sizeof(node_t) * nn);
    if (!f || !P || !df || !dP || !Phi || !dPhi || !nodes) return -2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) node_params(&L, p, x, y, &nodes[y * nx + x]);
    init_populations(&L, p, f);
    if (df0) {
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (is_solid(p, x, y)) continue;
                size_t k = (size_t)y * nx + x;
                for (int j = 0; j < 2 * Q; ++j) df[k * 2 * Q + j] = df0[k * 2 * Q + j];
            }
    }
    for (int n = 0; n < p->N; ++n) {
        memset(P, 0, sizeof(double) * npop);
        memset(dP, 0, sizeof(double) * npop);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (is_solid(p, x, y)) continue;
                double Pi[9][9], dfeq[9];
                size_t k = (size_t)y * nx + x;
                const node_t* nd = &nodes[k];
                const double *fu = f + (k * 2) * Q, *fv = f + (k * 2 + 1) * Q;
                const double *dfu = df + (k * 2) * Q, *dfv = df + (k * 2 + 1) * Q;
                double *dPu = dP + (k * 2) * Q, *dPv = dP + (k * 2 + 1) * Q;
                state_t st;
                double Phi_prev = Phi[k], dPhi_prev = dPhi[k];
                collide_local(&L, p, nd, n, fu, fv, g_at(p, g, n, x, y), Phi_prev, P + (k * 2) * Q,
                              P + (k * 2 + 1) * Q, &st);
                /* tangent of the local map (LIBEG-V) */
                double dTu = 0.0, dTv = 0.0, djv[2] = {0.0, 0.0};
                for (int i = 0; i < Q; ++i) {
                    dTu += dfu[i];
                    dTv += dfv[i];
                    djv[0] += L.e[i][0] * dfv[i];
                    djv[1] += L.e[i][1] * dfv[i];
                }
                double dPh = p->r_vu * dTu + p->r_vv * dTv + g_at(p, dg, n, x, y);
                if (n == 0) dPhi_prev = dPh;
                double dG[2];
                grad_v(p, nd, dTv, djv, dPh, dG); /* G is linear in (j_v, v, Phi) */
                Pi_matrix(&L, p, nd->Ku, Pi);
                feq_lat(&L, dTu, nd->a, p->d_u, dfeq);
                mrt_collide(&L, Pi, dfu, dfeq, dPu);
                double dAG[2];
                for (int c = 0; c < 2; ++c)
                    dAG[c] = p->chi / p->tau *
                             ((nd->Ku[c][0] * st.G[0] + nd->Ku[c][1] * st.G[1]) * dTu +
                              (nd->Ku[c][0] * dG[0] + nd->Ku[c][1] * dG[1]) * st.Theta_u);
                for (int i = 0; i < Q; ++i)
                    dPu[i] += p->tau * L.w[i] / CS2 * (L.e[i][0] * dAG[0] + L.e[i][1] * dAG[1]);
                Pi_matrix(&L, p, nd->Kv, Pi);
                feq_lat(&L, dTv, nd->a, p->d_v, dfeq);
                mrt_collide(&L, Pi, dfv, dfeq, dPv);
                for (int i = 0; i < Q; ++i) {
                    double src = p->tau * nd->wt_v[i] * dPh;
                    if (p->source_order != 1) src += 0.5 * p->tau * nd->wt_v[i] * (dPh - dPhi_prev);
                    dPv[i] += src;
                }
                Phi[k] = st.Phi;
                dPhi[k] = dPh;
            }
        stream_pull(&L, p, P, f);
        stream_pull(&L, p, dP, df);
    }
    double *u = malloc(sizeof(double) * nn), *du = malloc(sizeof(double) * nn);
    double* dv = malloc(sizeof(double) * nn);
    macro_fields(p, f, u, NULL);
    macro_fields(p, df, du, dv);
    double s = 0.0;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            size_t k = (size_t)y * nx + x;
            s += (u[k] - p->u_tgt[k]) * du[k];
        }
    if (g && dg)
        for (int n = 0; n < p->N; ++n)
            for (int y = 0; y < ny; ++y)
                for (int x = 0; x < nx; ++x) {
                    int c = ctrl_index(p, x, y);
                    if (c < 0) continue;
                    size_t idx = (size_t)n * p->cnx * p->cny + c;
                    s += 2.0 * p->alpha * g[idx] * dg[idx];
                }
    if (duN) memcpy(duN, du, sizeof(double) * nn);
    if (dvN) memcpy(dvN, dv, sizeof(double) * nn);
    if (dJ) *dJ = s;
    free(f); free(P); free(df); free(dP); free(Phi); free(dPhi); free(nodes);
    free(u); free(du); free(dv);
    return 0;
}

/* ------------------------------------------------------- AMRT adjoint */

/* One node of the AMRT adjoint step at step n (Sec. 3.2.1, eqs. CAE, AEDs,
 * CAE-L), the exact transpose of collide_local: from the pulled adjoint
 * populations rho (rho_i(x) = psi^{n+1}_i(x + e_i)) and the node's forward
 * state at step n (pre-collision populations f, Phi = Phi^n), the adjoint
 * populations psi^n of the node, sigma^n = sum_i rho_v,i w~_i, and lambda_Phi,
 * the adjoint of Phi^n (its use at step n and, when has_next, with
 * c'_{n+1} sigma^{n+1} at step n + 1), which is dJ/dg^n without the penalty. */
static void adjoint_local(const lattice_t* L, const or_problem* p, const node_t* nd, int n, const double* fu,
                          const double* fv, double Phi, const double* ru, const double* rv, int has_next,
                          double sigma_next, double* psi_u_out, double* psi_v_out, double* sigma_out,
                          double* adj_Phi_out) {
    const int Q = L->Q;
    double Pi[9][9], mt[9], psi_u[9], psi_v[9];
    /* forward state at (x, n) */
    double Tu = 0.0, Tv = 0.0, jv[2] = {0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        Tu += fu[i];
        Tv += fv[i];
        jv[0] += L->e[i][0] * fv[i];
        jv[1] += L->e[i][1] * fv[i];
    }
    double G[2];
    grad_v(p, nd, Tv, jv, Phi, G);

    /* AMRT collision: psi - Lambda^T (psi - psi^eq), with the
     * moment-space adjoint equilibrium m~^eq_i = T = sum_j w_j aleph_j m~_j */
    Pi_matrix(L, p, nd->Ku, Pi);
    mrt_collide_T(L, Pi, ru, mt);
    double Tcal = 0.0;
    for (int j = 0; j < Q; ++j) Tcal += L->w[j] * nd->aleph_u[j] * mt[j];
    for (int i = 0; i < Q; ++i) psi_u[i] = ru[i] - mt[i] + Tcal;
    Pi_matrix(L, p, nd->Kv, Pi);
    mrt_collide_T(L, Pi, rv, mt);
    Tcal = 0.0;
    for (int j = 0; j < Q; ++j) Tcal += L->w[j] * nd->aleph_v[j] * mt[j];
    for (int i = 0; i < Q; ++i) psi_v[i] = rv[i] - mt[i] + Tcal;

    /* coupling terms sum_k psi_k dR_k/dphi_i (CAE-L) */
    double adj_Tu = 0.0, adj_Tv = 0.0, adj_Phi = 0.0, adj_jv[2];
    /* R_u = tau S_u,  tau S_u,k = tau w_k/Cs^2 e_k . (K_u G) chi Tu / tau */
    double Y[2] = {0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        Y[0] += ru[i] * L->w[i] / CS2 * L->e[i][0];
        Y[1] += ru[i] * L->w[i] / CS2 * L->e[i][1];
    }
    double KG[2] = {nd->Ku[0][0] * G[0] + nd->Ku[0][1] * G[1], nd->Ku[1][0] * G[0] + nd->Ku[1][1] * G[1]};
    adj_Tu += p->chi * (Y[0] * KG[0] + Y[1] * KG[1]);
    double adj_G[2] = {p->chi * Tu * (nd->Ku[0][0] * Y[0] + nd->Ku[1][0] * Y[1]),
                       p->chi * Tu * (nd->Ku[0][1] * Y[0] + nd->Ku[1][1] * Y[1])};
    /* G = -(K_v (j_v - a v)/tau + K_v a Phi / 2) / (d_v Cs^2) */
    double KtG[2] = {nd->Kv[0][0] * adj_G[0] + nd->Kv[1][0] * adj_G[1],
                     nd->Kv[0][1] * adj_G[0] + nd->Kv[1][1] * adj_G[1]};
    double sc = 1.0 / (p->d_v * CS2);
    adj_jv[0] = -KtG[0] * sc / p->tau;
    adj_jv[1] = -KtG[1] * sc / p->tau;
    adj_Tv += (nd->a[0] * KtG[0] + nd->a[1] * KtG[1]) * sc / p->tau;
    adj_Phi += -0.5 * (nd->a[0] * KtG[0] + nd->a[1] * KtG[1]) * sc;
    /* R_v = w~ (c_n Phi^n + c'_n Phi^{n-1}) and the use of Phi^n at step n+1 */
    double sigma = 0.0;
    for (int i = 0; i < Q; ++i) sigma += rv[i] * nd->wt_v[i];
    adj_Phi += c_now(p, n) * sigma;
    if (has_next) adj_Phi += c_prev(p, n + 1) * sigma_next;
    *sigma_out = sigma;
    /* Phi = r_vu u + r_vv v + g */
    adj_Tu += p->r_vu * adj_Phi;
    adj_Tv += p->r_vv * adj_Phi;
    *adj_Phi_out = adj_Phi;
    for (int i = 0; i < Q; ++i) {
        psi_u_out[i] = psi_u[i] + adj_Tu;
        psi_v_out[i] = psi_v[i] + adj_Tv + L->e[i][0] * adj_jv[0] + L->e[i][1] * adj_jv[1];
    }
}

int or_adjoint(const or_problem* p, const double* g, const double* seed_u, const double* seed_v,
               double* dJdg, double* psi0, double* J) {
    lattice_t L;
    if (lattice_init(&L, p->Q)) return -1;
    int Q = p->Q, nx = p->nx, ny = p->ny, N = p->N;
    size_t nn = (size_t)nx * ny, npop = nn * 2 * Q, nc = (size_t)p->cnx * p->cny;
    double* traj = malloc(sizeof(double) * npop * (size_t)N);
    double* Phi_traj = malloc(sizeof(double) * nn * (size_t)N);
    double* fN = malloc(sizeof(double) * npop);
    double* psi = calloc(npop, sizeof(double));
    double* rho = calloc(npop, sizeof(double));
    double* sigma_next = calloc(nn, sizeof(double));
    double* sigma_now = calloc(nn, sizeof(double));
    double* u = malloc(sizeof(double) * nn);
    node_t* nodes = malloc(sizeof(node_t) * nn);
    if (!traj || !Phi_traj || !fN || !psi || !rho || !sigma_next || !sigma_now || !u || !nodes) return -2;
    int rc = run_forward(p, g, fN, traj, Phi_traj, NULL, NULL, NULL);
    if (rc) return rc;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) node_params(&L, p, x, y, &nodes[y * nx + x]);
    macro_fields(p, fN, u, NULL);
    if (J) *J = terminal_cost(p, u) + control_penalty(p, g);

    /* final condition: psi_i(T) = d I0 / d phi_i  (CAE) */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            size_t k = (size_t)y * nx + x;
            double wu = seed_u ? seed_u[k] : (u[k] - p->u_tgt[k]);
            double wv = seed_v ? seed_v[k] : 0.0;
            for (int i = 0; i < Q; ++i) {
                psi[(k * 2) * Q + i] = wu;
                psi[(k * 2 + 1) * Q + i] = wv;
            }
        }
    if (dJdg) memset(dJdg, 0, sizeof(double) * nc * (size_t)N);

    for (int n = N - 1; n >= 0; --n) {
        /* streaming along -e_i, backward in time */
        stream_pull_T(&L, p, psi, rho);
        memset(psi, 0, sizeof(double) * npop);
        const double* f = traj + (size_t)n * npop;
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (is_solid(p, x, y)) continue;
                size_t k = (size_t)y * nx + x;
                const double *fu = f + (k * 2) * Q, *fv = f + (k * 2 + 1) * Q;
                const double *ru = rho + (k * 2) * Q, *rv = rho + (k * 2 + 1) * Q;
                double adj_Phi;
                adjoint_local(&L, p, &nodes[k], n, fu, fv, Phi_traj[(size_t)n * nn + k], ru, rv, n + 1 <= N - 1,
                              sigma_next[k], psi + (k * 2) * Q, psi + (k * 2 + 1) * Q, &sigma_now[k], &adj_Phi);
                int c = ctrl_index(p, x, y);
                if (c >= 0 && dJdg) {
                    double gv = g ? g[(size_t)n * nc + c] : 0.0;
                    dJdg[(size_t)n * nc + c] = adj_Phi + 2.0 * p->alpha * gv;
                }
            }
        double* t = sigma_next;
        sigma_next = sigma_now;
        sigma_now = t;
    }
    if (psi0) memcpy(psi0, psi, sizeof(double) * npop);
    free(traj); free(Phi_traj); free(fN); free(psi); free(rho);
    free(sigma_next); free(sigma_now); free(u); free(nodes);
    return 0;
}

/* ------------------------------------------------------ unit-test access */

int or_adjoint_node(const or_problem* p, int x, int y, int n, const double* f_u, const double* f_v, double g,
                    const double* rho_u, const double* rho_v, int has_next, double sigma_next, double* psi_u,
                    double* psi_v, double* sigma_out, double* lam_Phi) {
    lattice_t L;
    if (lattice_init(&L, p->Q)) return -1;
    if (x < 0 || y < 0 || x >= p->nx || y >= p->ny) return -3;
    node_t nd;
    node_params(&L, p, x, y, &nd);
    double Tu = 0.0, Tv = 0.0;
    for (int i = 0; i < p->Q; ++i) {
        Tu += f_u[i];
        Tv += f_v[i];
    }
    const double Phi = p->r_vu * Tu + p->r_vv * Tv + g; /* as collide_local forms Phi^n */
    adjoint_local(&L, p, &nd, n, f_u, f_v, Phi, rho_u, rho_v, has_next, sigma_next, psi_u, psi_v, sigma_out,
                  lam_Phi);
    return 0;
}

int or_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int or_lattice(int Q, int* e, double* w, double* M, double* Minv) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    for (int i = 0; i < Q; ++i) {
        if (e) {
            e[2 * i] = L.e[i][0];
            e[2 * i + 1] = L.e[i][1];
        }
        if (w) w[i] = L.w[i];
        for (int j = 0; j < Q; ++j) {
            if (M) M[i * Q + j] = L.M[i][j];
            if (Minv) Minv[i * Q + j] = L.Minv[i][j];
        }
    }
    return 0;
}

int or_feq(int Q, double Theta, const double a[2], double d, double* out) {
    lattice_t L;
    if (lattice_init(&L, Q)) return -1;
    double aa[2] = {a ? a[0] : 0.0, a ? a[1] : 0.0};
    feq_lat(&L, Theta, aa, d, out);
    return 0;
}

/* ------------------------------------------------- continuous adjoint */

/* The continuous adjoint system (see mrt_oracle.h), time-reversed, solved by
 * the forward MRT scheme of Sec. 3.1 with:
 *   - convection velocity -a for both adjoint species (a.grad X = div(a X)
 *     for the solenoidal fields used here);
 *   - the terms chi grad v . grad u~ + r_vu v~ (for u~) and r_vv v~ (for v~)
 *     as first-order sources tau w~_i Phi (no (tau/2) time-derivative term);
 *   - -div(chi u grad u~) in the v~ equation as the chemotaxis-type source
 *     (w_i / Cs^2) chi u e_i . (K_v grad u~), the construction the forward
 *     uses for -div(chi u grad v);
 *   - grad u~ from u~'s first non-equilibrium moment,
 *     -K_u (j~_u + a u~) / (tau d_u Cs^2) (relation C146 without the source
 *     correction, since that source depends on grad u~ itself);
 *   - u, grad v at forward step n (the collision of step n) paired with the
 *     adjoint step from t_{n+1} back to t_n.
 * At s = 0 the adjoint populations are phi^eq(u~(0), -a) and 0. */
int or_cadjoint(const or_problem* p, const double* g, double* dJdg, double* J) {
    lattice_t L;
    if (lattice_init(&L, p->Q)) return -1;
    int Q = p->Q, nx = p->nx, ny = p->ny, N = p->N;
    size_t nn = (size_t)nx * ny, npop = nn * 2 * Q;
    double* fN = calloc(npop, sizeof(double));
    double* traj = calloc((size_t)N * npop, sizeof(double));
    double* fa = calloc(npop, sizeof(double));
    double* Pa = calloc(npop, sizeof(double));
    node_t* nodes = malloc(sizeof(node_t) * nn);
    double* wtu = malloc(sizeof(double) * nn * 9);
    double* wtv = malloc(sizeof(double) * nn * 9);
    if (!fN || !traj || !fa || !Pa || !nodes || !wtu || !wtv) return -2;
    int rc = run_forward(p, g, fN, traj, NULL, NULL, NULL, NULL);
    if (rc) return rc;
    double* u = malloc(sizeof(double) * nn);
    macro_fields(p, fN, u, NULL);
    if (J) *J = terminal_cost(p, u) + control_penalty(p, g);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            size_t k = (size_t)y * nx + x;
            node_params(&L, p, x, y, &nodes[k]);
            /* w~_i = w_i (1 + V.e_i / Cs^2), V = (I - K/2)(-a), per adjoint species */
            for (int sp = 0; sp < 2; ++sp) {
                double (*K)[2] = sp == 0 ? nodes[k].Ku : nodes[k].Kv;
                double am[2] = {-nodes[k].a[0], -nodes[k].a[1]};
                double V[2] = {am[0] - 0.5 * (K[0][0] * am[0] + K[0][1] * am[1]),
                               am[1] - 0.5 * (K[1][0] * am[0] + K[1][1] * am[1])};
                double* wt = (sp == 0 ? wtu : wtv) + k * 9;
                for (int i = 0; i < Q; ++i) wt[i] = L.w[i] * (1.0 + (V[0] * L.e[i][0] + V[1] * L.e[i][1]) / CS2);
            }
        }
    /* initial adjoint populations */
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (is_solid(p, x, y)) continue;
            size_t k = (size_t)y * nx + x;
            double am[2] = {-nodes[k].a[0], -nodes[k].a[1]};
            feq_lat(&L, u[k] - p->u_tgt[k], am, p->d_u, fa + (k * 2) * Q);
        }
    size_t nctrl = (size_t)p->cnx * p->cny;
    memset(dJdg, 0, sizeof(double) * (size_t)N * nctrl);
    for (int n = N - 1; n >= 0; --n) {
        const double* f = traj + (size_t)n * npop; /* forward pre-collision state of step n */
        memset(Pa, 0, sizeof(double) * npop);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                if (is_solid(p, x, y)) continue;
                double Pi[9][9], feq[9];
                size_t k = (size_t)y * nx + x;
                const node_t* nd = &nodes[k];
                /* forward quantities of step n: u^n and grad v^n */
                state_t st;
                double Ptmp[18];
                collide_local(&L, p, nd, n, f + (k * 2) * Q, f + (k * 2 + 1) * Q, g_at(p, g, n, x, y), 0.0,
                              Ptmp, Ptmp + 9, &st);
                const double* au = fa + (k * 2) * Q;
                const double* av = fa + (k * 2 + 1) * Q;
                double ut = 0.0, vt = 0.0, ju[2] = {0.0, 0.0};
                for (int i = 0; i < Q; ++i) {
                    ut += au[i];
                    vt += av[i];
                    ju[0] += L.e[i][0] * au[i];
                    ju[1] += L.e[i][1] * au[i];
                }
                double am[2] = {-nd->a[0], -nd->a[1]};
                double r[2] = {(ju[0] - am[0] * ut) / p->tau, (ju[1] - am[1] * ut) / p->tau};
                double gu[2];
                for (int c = 0; c < 2; ++c) gu[c] = -(nd->Ku[c][0] * r[0] + nd->Ku[c][1] * r[1]) / (p->d_u * CS2);
                int c = ctrl_index(p, x, y);
                if (c >= 0) dJdg[(size_t)n * nctrl + c] = 2.0 * p->alpha * g_at(p, g, n, x, y) + vt;
                double Phu = p->chi * (st.G[0] * gu[0] + st.G[1] * gu[1]) + p->r_vu * vt;
                double Phv = p->r_vv * vt;
                double* Pu = Pa + (k * 2) * Q;
                double* Pv = Pa + (k * 2 + 1) * Q;
                Pi_matrix(&L, p, nd->Ku, Pi);
                feq_lat(&L, ut, am, p->d_u, feq);
                mrt_collide(&L, Pi, au, feq, Pu);
                for (int i = 0; i < Q; ++i) Pu[i] += p->tau * wtu[k * 9 + i] * Phu;
                Pi_matrix(&L, p, nd->Kv, Pi);
                feq_lat(&L, vt, am, p->d_v, feq);
                mrt_collide(&L, Pi, av, feq, Pv);
                double F[2];
                for (int cc = 0; cc < 2; ++cc)
                    F[cc] = p->chi * st.Theta_u * (nd->Kv[cc][0] * gu[0] + nd->Kv[cc][1] * gu[1]);
                for (int i = 0; i < Q; ++i)
                    Pv[i] += p->tau * wtv[k * 9 + i] * Phv + L.w[i] / CS2 * (L.e[i][0] * F[0] + L.e[i][1] * F[1]);
            }
        stream_pull(&L, p, Pa, fa);
    }
    /* controlled nodes that are solid carry no gradient */
    free(fN);
    free(traj);
    free(fa);
    free(Pa);
    free(nodes);
    free(wtu);
    free(wtv);
    free(u);
    return 0;
}

/* ===================================================================
 * Three species (u, v, w): the attraction-repulsion chemotaxis model with
 * a logistic source (the ARC example of Sec. 2.2, a case of the paper's
 * three-equation system eq. ReacDiff), solved by the same coupled MRT
 * scheme of Sec. 3.1 (eq. LBE with S, PhiS, phieq) and differentiated by the
 * exact discrete adjoint of Sec. 3.2.1.  See mrt_oracle.h (or3_problem).
 *   Phi_u = a1 u - a2 u^2, Phi_v = b1 u - b2 v - b3 u v, Phi_w = c1 u - c2 w,
 *   and the control g added to Phi_v or Phi_w;
 *   S_u,i = (w_i/Cs^2) e_i . (K_u (chi1 u G_v + chi2 u G_w)) (eq. S with
 *   D_{u,1} = chi1 u I toward v and D_{u,2} = chi2 u I toward w);
 *   G_Theta the local gradient of Theta = v, w from its non-equilibrium flux
 *   (the reading of C146 used for v in the two-species model).
 * Populations [ny][nx][3][Q] (species u, v, w), periodic grid, D2Q9.
 * =================================================================== */

typedef struct {
    double K[3][2][2];   /* relaxation blocks of u, v, w */
    double a[2];
    double aleph[3][9];  /* adjoint-equilibrium weights per species */
    double wt[3][9];     /* w~_i = w_i (1 + V_Theta.e_i / Cs^2), V_Theta = (I - K_Theta/2) a */
} node3_t;

static void Pi_rates(const double s[7], const double K[2][2], double Pi[9][9]) {
    memset(Pi, 0, sizeof(double) * 81);
    Pi[0][0] = s[0];
    Pi[1][1] = s[1];
    Pi[2][2] = s[2];
    Pi[3][3] = K[0][0];
    Pi[3][5] = K[0][1];
    Pi[4][4] = s[3];
    Pi[5][3] = K[1][0];
    Pi[5][5] = K[1][1];
    Pi[6][6] = s[4];
    Pi[7][7] = s[5];
    Pi[8][8] = s[6];
}

static void node3_params(const lattice_t* L, const or3_problem* p, int x, int y, node3_t* nd) {
    int k = y * p->nx + x;
    const double* D[3] = {p->Du, p->Dv, p->Dw};
    nd->a[0] = p->a ? p->a[2 * k] : 0.0;
    nd->a[1] = p->a ? p->a[2 * k + 1] : 0.0;
    for (int sp = 0; sp < 3; ++sp) {
        K_from_D(D[sp] + 3 * k, p->d, p->tau, nd->K[sp]);
        aleph_lat(L, nd->a, p->d, nd->aleph[sp]);
        double V[2];
        for (int c = 0; c < 2; ++c)
            V[c] = nd->a[c] - 0.5 * (nd->K[sp][c][0] * nd->a[0] + nd->K[sp][c][1] * nd->a[1]);
        for (int i = 0; i < L->Q; ++i)
            nd->wt[sp][i] = L->w[i] * (1.0 + (V[0] * L->e[i][0] + V[1] * L->e[i][1]) / CS2);
    }
}

static double c3_now(const or3_problem* p, int n) { return (p->source_order == 1 || n == 0) ? p->tau : 1.5 * p->tau; }
static double c3_prev(const or3_problem* p, int n) { return (p->source_order == 1 || n == 0) ? 0.0 : -0.5 * p->tau; }

/* reaction/control sources (the kinetics of the ARC example) */
static void phi3(const or3_problem* p, double Tu, double Tv, double Tw, double g, double Phi[3]) {
    Phi[0] = p->a1 * Tu - p->a2 * Tu * Tu;
    Phi[1] = p->b1 * Tu - p->b2 * Tv - p->b3 * Tu * Tv + (p->ctrl_species == 1 ? g : 0.0);
    Phi[2] = p->c1 * Tu - p->c2 * Tw + (p->ctrl_species == 2 ? g : 0.0);
}

/* local gradient of a species from its first non-equilibrium moment (C146 reading) */
static void grad3(const or3_problem* p, const double K[2][2], const double a[2], double T, const double j[2],
                  double Phi, double G[2]) {
    double r[2] = {(j[0] - a[0] * T) / p->tau, (j[1] - a[1] * T) / p->tau};
    for (int c = 0; c < 2; ++c)
        G[c] = -(K[c][0] * r[0] + K[c][1] * r[1] + 0.5 * (K[c][0] * a[0] + K[c][1] * a[1]) * Phi) / (p->d * CS2);
}

typedef struct {
    double T[3], Phi[3], Gv[2], Gw[2];
} state3_t;

/* one collision of the three species at a node: f[3][Q] -> P[3][Q] */
static void collide3(const lattice_t* L, const or3_problem* p, const node3_t* nd, int n, const double* f,
                     double g, const double Phi_prev[3], double* P, state3_t* st) {
    int Q = L->Q;
    double T[3] = {0, 0, 0}, j[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int sp = 0; sp < 3; ++sp)
        for (int i = 0; i < Q; ++i) {
            T[sp] += f[sp * Q + i];
            j[sp][0] += L->e[i][0] * f[sp * Q + i];
            j[sp][1] += L->e[i][1] * f[sp * Q + i];
        }
    double Phi[3], Pp[3];
    phi3(p, T[0], T[1], T[2], g, Phi);
    for (int sp = 0; sp < 3; ++sp) Pp[sp] = (n == 0) ? Phi[sp] : Phi_prev[sp];
    double Gv[2], Gw[2];
    grad3(p, nd->K[1], nd->a, T[1], j[1], Phi[1], Gv);
    grad3(p, nd->K[2], nd->a, T[2], j[2], Phi[2], Gw);
    double Pi[9][9], feq[9];
    for (int sp = 0; sp < 3; ++sp) {
        Pi_rates(p->s, nd->K[sp], Pi);
        feq_lat(L, T[sp], nd->a, p->d, feq);
        mrt_collide(L, Pi, f + sp * Q, feq, P + sp * Q);
        for (int i = 0; i < Q; ++i) {
            double src = p->tau * nd->wt[sp][i] * Phi[sp];
            if (p->source_order != 1) src += 0.5 * p->tau * nd->wt[sp][i] * (Phi[sp] - Pp[sp]);
            P[sp * Q + i] += src;
        }
    }
    /* tau S_u: chemotactic fluxes toward v (chi1) and w (chi2) */
    double F[2];
    for (int c = 0; c < 2; ++c) F[c] = p->chi1 * T[0] * Gv[c] + p->chi2 * T[0] * Gw[c];
    double KF[2] = {nd->K[0][0][0] * F[0] + nd->K[0][0][1] * F[1], nd->K[0][1][0] * F[0] + nd->K[0][1][1] * F[1]};
    for (int i = 0; i < Q; ++i) P[i] += L->w[i] / CS2 * (L->e[i][0] * KF[0] + L->e[i][1] * KF[1]);
    if (st) {
        for (int sp = 0; sp < 3; ++sp) {
            st->T[sp] = T[sp];
            st->Phi[sp] = Phi[sp];
        }
        st->Gv[0] = Gv[0];
        st->Gv[1] = Gv[1];
        st->Gw[0] = Gw[0];
        st->Gw[1] = Gw[1];
    }
}

static void stream3(const lattice_t* L, const or3_problem* p, const double* P, double* f, int adjoint) {
    int Q = L->Q, nx = p->nx, ny = p->ny;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x)
            for (int sp = 0; sp < 3; ++sp)
                for (int i = 0; i < Q; ++i) {
                    int sx = adjoint ? L->e[i][0] : -L->e[i][0], sy = adjoint ? L->e[i][1] : -L->e[i][1];
                    int xs = (x + sx + nx) % nx, ys = (y + sy + ny) % ny;
                    f[((size_t)(y * nx + x) * 3 + sp) * Q + i] = P[((size_t)(ys * nx + xs) * 3 + sp) * Q + i];
                }
}

static int run3_forward(const or3_problem* p, const double* g, double* fN, double* traj, double* Phi_traj,
                        double* trace) {
    lattice_t L;
    if (lattice_init(&L, 9)) return -1;
    int Q = 9, nx = p->nx, ny = p->ny;
    size_t nn = (size_t)nx * ny, npop = nn * 3 * Q;
    double* f = calloc(npop, sizeof(double));
    double* P = calloc(npop, sizeof(double));
    double* Phi = calloc(nn * 3, sizeof(double));
    double* Th = calloc(nn * 3, sizeof(double));
    node3_t* nodes = malloc(sizeof(node3_t) * nn);
    if (!f || !P || !Phi || !Th || !nodes) return -2;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) node3_params(&L, p, x, y, &nodes[y * nx + x]);
    const double* init[3] = {p->u0, p->v0, p->w0};
    for (size_t k = 0; k < nn; ++k)
        for (int sp = 0; sp < 3; ++sp) feq_lat(&L, init[sp][k], nodes[k].a, p->d, f + (k * 3 + sp) * Q);
    for (int n = 0; n < p->N; ++n) {
        if (traj) memcpy(traj + (size_t)n * npop, f, sizeof(double) * npop);
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = (size_t)y * nx + x;
                state3_t st;
                double gv = g ? g[(size_t)n * nn + k] : 0.0;
                collide3(&L, p, &nodes[k], n, f + k * 3 * Q, gv, Phi + 3 * k, P + k * 3 * Q, &st);
                for (int sp = 0; sp < 3; ++sp) {
                    Phi[3 * k + sp] = st.Phi[sp];
                    Th[3 * k + sp] = st.T[sp];
                }
            }
        if (Phi_traj) memcpy(Phi_traj + (size_t)n * nn * 3, Phi, sizeof(double) * nn * 3);
        if (trace) /* per step: mass of u, v, w before collision, then sum of Phi_u, Phi_v, Phi_w */
            for (int sp = 0; sp < 3; ++sp) {
                double m = 0.0, s = 0.0;
                for (size_t k = 0; k < nn; ++k) {
                    m += Th[3 * k + sp];
                    s += Phi[3 * k + sp];
                }
                trace[(size_t)n * 6 + sp] = m;
                trace[(size_t)n * 6 + 3 + sp] = s;
            }
        stream3(&L, p, P, f, 0);
    }
    memcpy(fN, f, sizeof(double) * npop);
    free(f);
    free(P);
    free(Phi);
    free(Th);
    free(nodes);
    return 0;
}

static double cost3(const or3_problem* p, const double* fN, const double* g, double* uvw) {
    size_t nn = (size_t)p->nx * p->ny;
    double s = 0.0, pen = 0.0;
    for (size_t k = 0; k < nn; ++k) {
        double T[3] = {0, 0, 0};
        for (int sp = 0; sp < 3; ++sp)
            for (int i = 0; i < 9; ++i) T[sp] += fN[(k * 3 + sp) * 9 + i];
        if (uvw)
            for (int sp = 0; sp < 3; ++sp) uvw[sp * nn + k] = T[sp];
        double d = T[0] - p->u_tgt[k];
        s += 0.5 * d * d;
    }
    if (g)
        for (size_t q = 0; q < (size_t)p->N * nn; ++q) pen += g[q] * g[q];
    return s + p->alpha * pen;
}

int or3_forward(const or3_problem* p, const double* g, double* J, double* uvwN) {
    size_t nn = (size_t)p->nx * p->ny;
    double* fN = malloc(sizeof(double) * nn * 27);
    if (!fN) return -2;
    int rc = run3_forward(p, g, fN, NULL, NULL, NULL);
    if (rc) return rc;
    double c = cost3(p, fN, g, uvwN);
    if (J) *J = c;
    free(fN);
    return 0;
}

int or3_forward_trace(const or3_problem* p, const double* g, double* trace) {
    size_t nn = (size_t)p->nx * p->ny;
    double* fN = malloc(sizeof(double) * nn * 27);
    if (!fN) return -2;
    int rc = run3_forward(p, g, fN, NULL, NULL, trace);
    free(fN);
    return rc;
}

/* Tangent-linear model of the three-species forward solve along dg (and df0,
 * [ny][nx][3][Q], may be NULL): duvwN [3][ny][nx] and the derivative dJ. */
int or3_tlm(const or3_problem* p, const double* g, const double* dg, const double* df0, double* duvwN, double* dJ) {
    lattice_t L;
    if (lattice_init(&L, 9)) return -1;
    int Q = 9, nx = p->nx, ny = p->ny;
    size_t nn = (size_t)nx * ny, npop = nn * 3 * Q;
    double *f = calloc(npop, sizeof(double)), *P = calloc(npop, sizeof(double));
    double *df = calloc(npop, sizeof(double)), *dP = calloc(npop, sizeof(double));
    double *Phi = calloc(nn * 3, sizeof(double)), *dPhi = calloc(nn * 3, sizeof(double));
    node3_t* nodes = malloc(sizeof(node3_t) * nn);
    if (!f || !P || !df || !dP || !Phi || !dPhi || !nodes) return -2;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) node3_params(&L, p, x, y, &nodes[y * nx + x]);
    const double* init[3] = {p->u0, p->v0, p->w0};
    for (size_t k = 0; k < nn; ++k)
        for (int sp = 0; sp < 3; ++sp) feq_lat(&L, init[sp][k], nodes[k].a, p->d, f + (k * 3 + sp) * Q);
    if (df0) memcpy(df, df0, sizeof(double) * npop);
    for (int n = 0; n < p->N; ++n) {
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = (size_t)y * nx + x;
                const node3_t* nd = &nodes[k];
                state3_t st;
                double gv = g ? g[(size_t)n * nn + k] : 0.0;
                double dgv = dg ? dg[(size_t)n * nn + k] : 0.0;
                collide3(&L, p, nd, n, f + k * 3 * Q, gv, Phi + 3 * k, P + k * 3 * Q, &st);
                /* tangent of the local map */
                const double* dfk = df + k * 3 * Q;
                double* dPk = dP + k * 3 * Q;
                double dT[3] = {0, 0, 0}, dj[3][2] = {{0, 0}, {0, 0}, {0, 0}};
                for (int sp = 0; sp < 3; ++sp)
                    for (int i = 0; i < Q; ++i) {
                        dT[sp] += dfk[sp * Q + i];
                        dj[sp][0] += L.e[i][0] * dfk[sp * Q + i];
                        dj[sp][1] += L.e[i][1] * dfk[sp * Q + i];
                    }
                const double Tu = st.T[0], Tv = st.T[1];
                double dPh[3];
                dPh[0] = (p->a1 - 2.0 * p->a2 * Tu) * dT[0];
                dPh[1] = (p->b1 - p->b3 * Tv) * dT[0] - (p->b2 + p->b3 * Tu) * dT[1] + (p->ctrl_species == 1 ? dgv : 0.0);
                dPh[2] = p->c1 * dT[0] - p->c2 * dT[2] + (p->ctrl_species == 2 ? dgv : 0.0);
                double dPp[3];
                for (int sp = 0; sp < 3; ++sp) dPp[sp] = (n == 0) ? dPh[sp] : dPhi[3 * k + sp];
                double dGv[2], dGw[2];
                grad3(p, nd->K[1], nd->a, dT[1], dj[1], dPh[1], dGv); /* G is linear in (j, T, Phi) */
                grad3(p, nd->K[2], nd->a, dT[2], dj[2], dPh[2], dGw);
                double Pi[9][9], dfeq[9];
                for (int sp = 0; sp < 3; ++sp) {
                    Pi_rates(p->s, nd->K[sp], Pi);
                    feq_lat(&L, dT[sp], nd->a, p->d, dfeq);
                    mrt_collide(&L, Pi, dfk + sp * Q, dfeq, dPk + sp * Q);
                    for (int i = 0; i < Q; ++i) {
                        double src = p->tau * nd->wt[sp][i] * dPh[sp];
                        if (p->source_order != 1) src += 0.5 * p->tau * nd->wt[sp][i] * (dPh[sp] - dPp[sp]);
                        dPk[sp * Q + i] += src;
                    }
                }
                double dF[2];
                for (int c = 0; c < 2; ++c)
                    dF[c] = (p->chi1 * st.Gv[c] + p->chi2 * st.Gw[c]) * dT[0] +
                            Tu * (p->chi1 * dGv[c] + p->chi2 * dGw[c]);
                double dKF[2] = {nd->K[0][0][0] * dF[0] + nd->K[0][0][1] * dF[1],
                                 nd->K[0][1][0] * dF[0] + nd->K[0][1][1] * dF[1]};
                for (int i = 0; i < Q; ++i) dPk[i] += L.w[i] / CS2 * (L.e[i][0] * dKF[0] + L.e[i][1] * dKF[1]);
                for (int sp = 0; sp < 3; ++sp) {
                    Phi[3 * k + sp] = st.Phi[sp];
                    dPhi[3 * k + sp] = dPh[sp];
                }
            }
        stream3(&L, p, P, f, 0);
        stream3(&L, p, dP, df, 0);
    }
    double s = 0.0;
    for (size_t k = 0; k < nn; ++k) {
        double T[3] = {0, 0, 0}, dT[3] = {0, 0, 0};
        for (int sp = 0; sp < 3; ++sp)
            for (int i = 0; i < Q; ++i) {
                T[sp] += f[(k * 3 + sp) * Q + i];
                dT[sp] += df[(k * 3 + sp) * Q + i];
            }
        if (duvwN)
            for (int sp = 0; sp < 3; ++sp) duvwN[sp * nn + k] = dT[sp];
        s += (T[0] - p->u_tgt[k]) * dT[0];
    }
    if (g && dg)
        for (size_t q = 0; q < (size_t)p->N * nn; ++q) s += 2.0 * p->alpha * g[q] * dg[q];
    if (dJ) *dJ = s;
    free(f); free(P); free(df); free(dP); free(Phi); free(dPhi); free(nodes);
    return 0;
}

/* Exact discrete adjoint of the three-species forward solve.  seeds [3][ny][nx]
 * (adjoints of u^N, v^N, w^N), NULL meaning (u^N - u_tgt, 0, 0); with seeds the
 * gradient is that of sum(seed . uvw^N) + alpha ||g||^2.  dJdg [N][ny][nx];
 * psi0 [ny][nx][3][Q] (may be NULL); J (may be NULL). */
/* One node of the three-species AMRT step at step n, the exact transpose of
 * collide3: from the pulled adjoint populations rho ([3][Q], rho_i(x) =
 * psi^{n+1}_i(x + e_i)) and the node's forward state at step n (pre-collision
 * populations f [3][Q], Phi = Phi^n [3]), the node's adjoint populations psi
 * [3][Q], sigma^n [3] and aPhi [3], the adjoint of each species' Phi^n (its
 * use at step n and, when has_next, with c'_{n+1} sigma^{n+1} at step n + 1). */
static void adjoint3_local(const lattice_t* L, const or3_problem* p, const node3_t* nd, int n, const double* fk,
                           const double* Ph, const double* rk, int has_next, const double* sig_next,
                           double* psi_out, double* sig_out, double* aPhi) {
    const int Q = L->Q;
    /* forward state at (x, n) */
    double T[3] = {0, 0, 0}, j[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int sp = 0; sp < 3; ++sp)
        for (int i = 0; i < Q; ++i) {
            T[sp] += fk[sp * Q + i];
            j[sp][0] += L->e[i][0] * fk[sp * Q + i];
            j[sp][1] += L->e[i][1] * fk[sp * Q + i];
        }
    double Gv[2], Gw[2];
    grad3(p, nd->K[1], nd->a, T[1], j[1], Ph[1], Gv);
    grad3(p, nd->K[2], nd->a, T[2], j[2], Ph[2], Gw);
    /* transposed MRT collisions with the adjoint equilibrium broadcast */
    double out[27], Pi[9][9], mt[9];
    for (int sp = 0; sp < 3; ++sp) {
        Pi_rates(p->s, nd->K[sp], Pi);
        mrt_collide_T(L, Pi, rk + sp * Q, mt);
        double Tcal = 0.0;
        for (int i = 0; i < Q; ++i) Tcal += L->w[i] * nd->aleph[sp][i] * mt[i];
        for (int i = 0; i < Q; ++i) out[sp * Q + i] = rk[sp * Q + i] - mt[i] + Tcal;
    }
    /* adjoint of tau S_u = (w_i/Cs^2) e_i . K_u F,  F = u (chi1 G_v + chi2 G_w) */
    double Y[2] = {0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        Y[0] += rk[i] * L->w[i] / CS2 * L->e[i][0];
        Y[1] += rk[i] * L->w[i] / CS2 * L->e[i][1];
    }
    double aF[2] = {nd->K[0][0][0] * Y[0] + nd->K[0][1][0] * Y[1], nd->K[0][0][1] * Y[0] + nd->K[0][1][1] * Y[1]};
    double aT[3] = {0, 0, 0}, aj[3][2] = {{0, 0}, {0, 0}, {0, 0}};
    for (int sp = 0; sp < 3; ++sp) aPhi[sp] = 0.0;
    for (int c2 = 0; c2 < 2; ++c2) aT[0] += (p->chi1 * Gv[c2] + p->chi2 * Gw[c2]) * aF[c2];
    double aG[3][2];
    for (int c2 = 0; c2 < 2; ++c2) {
        aG[1][c2] = p->chi1 * T[0] * aF[c2];
        aG[2][c2] = p->chi2 * T[0] * aF[c2];
    }
    /* G_Theta = -(K (j - a T)/tau + K a Phi / 2) / (d Cs^2), Theta = v, w */
    for (int sp = 1; sp < 3; ++sp) {
        double KtG[2] = {nd->K[sp][0][0] * aG[sp][0] + nd->K[sp][1][0] * aG[sp][1],
                         nd->K[sp][0][1] * aG[sp][0] + nd->K[sp][1][1] * aG[sp][1]};
        double sc = 1.0 / (p->d * CS2);
        aj[sp][0] = -KtG[0] * sc / p->tau;
        aj[sp][1] = -KtG[1] * sc / p->tau;
        aT[sp] += (nd->a[0] * KtG[0] + nd->a[1] * KtG[1]) * sc / p->tau;
        aPhi[sp] += -0.5 * (nd->a[0] * KtG[0] + nd->a[1] * KtG[1]) * sc;
    }
    /* sources w~ (c_n Phi^n + c'_n Phi^{n-1}) and the use of Phi^n at step n+1 */
    for (int sp = 0; sp < 3; ++sp) {
        double sig = 0.0;
        for (int i = 0; i < Q; ++i) sig += rk[sp * Q + i] * nd->wt[sp][i];
        aPhi[sp] += c3_now(p, n) * sig;
        if (has_next) aPhi[sp] += c3_prev(p, n + 1) * sig_next[sp];
        sig_out[sp] = sig;
    }
    /* Phi_u = a1 u - a2 u^2, Phi_v = b1 u - b2 v - b3 u v (+ g), Phi_w = c1 u - c2 w (+ g) */
    aT[0] += (p->a1 - 2.0 * p->a2 * T[0]) * aPhi[0] + (p->b1 - p->b3 * T[1]) * aPhi[1] + p->c1 * aPhi[2];
    aT[1] += -(p->b2 + p->b3 * T[0]) * aPhi[1];
    aT[2] += -p->c2 * aPhi[2];
    for (int sp = 0; sp < 3; ++sp)
        for (int i = 0; i < Q; ++i)
            psi_out[sp * Q + i] =
                out[sp * Q + i] + aT[sp] + L->e[i][0] * aj[sp][0] + L->e[i][1] * aj[sp][1];
}

int or3_adjoint(const or3_problem* p, const double* g, const double* seeds, double* dJdg, double* psi0, double* J) {
    lattice_t L;
    if (lattice_init(&L, 9)) return -1;
    int Q = 9, nx = p->nx, ny = p->ny, N = p->N;
    size_t nn = (size_t)nx * ny, npop = nn * 3 * Q;
    double* traj = malloc(sizeof(double) * npop * (size_t)N);
    double* Phi_traj = malloc(sizeof(double) * nn * 3 * (size_t)N);
    double* fN = malloc(sizeof(double) * npop);
    double* psi = calloc(npop, sizeof(double));
    double* rho = calloc(npop, sizeof(double));
    double* sig_next = calloc(nn * 3, sizeof(double));
    double* sig_now = calloc(nn * 3, sizeof(double));
    double* uvw = malloc(sizeof(double) * nn * 3);
    node3_t* nodes = malloc(sizeof(node3_t) * nn);
    if (!traj || !Phi_traj || !fN || !psi || !rho || !sig_next || !sig_now || !uvw || !nodes) return -2;
    int rc = run3_forward(p, g, fN, traj, Phi_traj, NULL);
    if (rc) return rc;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) node3_params(&L, p, x, y, &nodes[y * nx + x]);
    double c = cost3(p, fN, g, uvw);
    if (J) *J = c;
    /* final condition: psi_Theta,i(T) = d I0 / d f_Theta,i */
    for (size_t k = 0; k < nn; ++k)
        for (int sp = 0; sp < 3; ++sp) {
            double wseed = seeds ? seeds[sp * nn + k] : (sp == 0 ? uvw[k] - p->u_tgt[k] : 0.0);
            for (int i = 0; i < Q; ++i) psi[(k * 3 + sp) * Q + i] = wseed;
        }
    if (dJdg) memset(dJdg, 0, sizeof(double) * nn * (size_t)N);
    for (int n = N - 1; n >= 0; --n) {
        stream3(&L, p, psi, rho, 1); /* streaming along -e_i, backward in time */
        const double* f = traj + (size_t)n * npop;
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                size_t k = (size_t)y * nx + x;
                double aPhi[3];
                adjoint3_local(&L, p, &nodes[k], n, f + k * 3 * Q, Phi_traj + ((size_t)n * nn + k) * 3,
                               rho + k * 3 * Q, n + 1 <= N - 1, sig_next + 3 * k, psi + k * 3 * Q,
                               sig_now + 3 * k, aPhi);
                if (dJdg) {
                    double gv = g ? g[(size_t)n * nn + k] : 0.0;
                    dJdg[(size_t)n * nn + k] = aPhi[p->ctrl_species] + 2.0 * p->alpha * gv;
                }
            }
        double* t = sig_next;
        sig_next = sig_now;
        sig_now = t;
    }
    if (psi0) memcpy(psi0, psi, sizeof(double) * npop);
    free(traj); free(Phi_traj); free(fN); free(psi); free(rho); free(sig_next); free(sig_now); free(uvw); free(nodes);
    return 0;
}

int or3_collide_node(const or3_problem* p, int x, int y, int n, const double* f, double g, const double* Phi_prev,
                     double* P, double* Phi_out) {
    lattice_t L;
    if (lattice_init(&L, 9)) return -1;
    if (x < 0 || y < 0 || x >= p->nx || y >= p->ny) return -3;
    node3_t nd;
    node3_params(&L, p, x, y, &nd);
    state3_t st;
    collide3(&L, p, &nd, n, f, g, Phi_prev, P, &st);
    for (int sp = 0; sp < 3; ++sp) Phi_out[sp] = st.Phi[sp];
    return 0;
}

int or3_adjoint_node(const or3_problem* p, int x, int y, int n, const double* f, double g, const double* rho,
                     int has_next, const double* sigma_next, double* psi, double* sigma_out, double* lam_Phi) {
    lattice_t L;
    if (lattice_init(&L, 9)) return -1;
    if (x < 0 || y < 0 || x >= p->nx || y >= p->ny) return -3;
    node3_t nd;
    node3_params(&L, p, x, y, &nd);
    double T[3] = {0, 0, 0};
    for (int sp = 0; sp < 3; ++sp)
        for (int i = 0; i < 9; ++i) T[sp] += f[sp * 9 + i];
    double Phi[3];
    phi3(p, T[0], T[1], T[2], g, Phi); /* as collide3 forms Phi^n */
    const double zero[3] = {0, 0, 0};
    adjoint3_local(&L, p, &nd, n, f, Phi, rho, has_next, sigma_next ? sigma_next : zero, psi, sigma_out, lam_Phi);
    return 0;
}
