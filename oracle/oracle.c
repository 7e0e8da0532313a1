/*
 * CPU oracle for the Wilson-Dirac operator of arXiv 1904.08616 and the CG solvers that
 * invert D^dag D.  TEST INFRASTRUCTURE: only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference legs load this library.  The CUDA library never
 * links, includes or calls it, and it shares no code with it.
 *
 * Everything is FP64, in plain loops over sites, directions, spin and colour, with no
 * blocking, no fusion and none of the rank-2 half-spinor shortcuts of the GPU kernels.
 *
 * Field storage (lexicographic site n = x + Lx*(y + Ly*(z + Lz*t)), mu = 0..3 <-> x,y,z,t):
 *   gauge  U[n][mu][row A][col B]  complex  (18 reals per link)
 *   spinor psi[n][spin alpha][colour A] complex (24 reals per site)
 *
 * Readings of points the paper leaves open (each is listed in the design notes):
 *   - hopping sign: the paper's literal "+1/2" (Eq. 1);
 *   - P^{-mu} = 1 - gamma_{mu+1}, P^{+mu} = 1 + gamma_{mu+1} (the paper calls them real
 *     4x4 constant matrices; no Hermitian basis makes all four real, so they are taken
 *     as 1 -/+ gamma in the chiral basis below);
 *   - the backward link U^dag(n - mu) of Eq. 1 is U_mu(n - mu)^dag;
 *   - boundary conditions periodic in all four directions.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* Threads over which the loops over output sites of lq_oracle_dslash and
 * lq_oracle_dslash_sites are split (1 = serial, the default).  Each output site is computed
 * by the same per-site routine and written by exactly one thread, so the results do not
 * depend on this number; it only serves to time the oracle on all host cores. */
static int g_threads = 1;

/* Cores the oracle can use: the OpenMP processor count, or 1 without OpenMP. */
int lq_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_num_procs();
#else
    return 1;
#endif
}

/* Sets the thread count (clamped to 1..lq_oracle_max_threads()); returns the count in use. */
int lq_oracle_set_threads(int n)
{
    const int mx = lq_oracle_max_threads();
    g_threads = n < 1 ? 1 : (n > mx ? mx : n);
    return g_threads;
}

/* ------------------------------------------------------------------------------------
 * Gamma matrices, chiral Euclidean basis (Hermitian, {g_mu, g_nu} = 2 delta):
 *   gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]   k = 1, 2, 3
 *   gamma_4 = [[0, 1], [1, 0]]
 * Direction mu = 0..3 uses gamma_{mu+1}.  gamma_5 = g1 g2 g3 g4 = diag(1, 1, -1, -1).
 * ---------------------------------------------------------------------------------- */
static void pauli(int k, cplx s[2][2])
{
    memset(s, 0, sizeof(cplx) * 4);
    if (k == 1) { s[0][1] = 1.0;  s[1][0] = 1.0; }
    if (k == 2) { s[0][1] = -I;   s[1][0] = I;   }
    if (k == 3) { s[0][0] = 1.0;  s[1][1] = -1.0; }
}

void lq_oracle_gamma(int mu, double *out_reals /* [4][4][re,im] */)
{
    cplx g[4][4];
    memset(g, 0, sizeof(g));
    if (mu == 3) {
        for (int i = 0; i < 2; ++i) { g[i][i + 2] = 1.0; g[i + 2][i] = 1.0; }
    } else {
        cplx s[2][2];
        pauli(mu + 1, s);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                g[i][j + 2] = -I * s[i][j];
                g[i + 2][j] = I * s[i][j];
            }
    }
    cplx *o = (cplx *)out_reals;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) o[4 * i + j] = g[i][j];
}

/* P[mu][sign] as a full 4x4 matrix: sign = -1 -> 1 - gamma, sign = +1 -> 1 + gamma. */
static void projector(int mu, int sign, cplx P[4][4])
{
    cplx g[4][4];
    lq_oracle_gamma(mu, (double *)g);
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) P[i][j] = (i == j ? 1.0 : 0.0) + (double)sign * g[i][j];
}

/* ------------------------------------------------------------------------------------
 * Lattice geometry.
 * ---------------------------------------------------------------------------------- */
static int64_t lex_index(const int32_t L[4], const int c[4])
{
    return (int64_t)c[0] + (int64_t)L[0] * ((int64_t)c[1] + (int64_t)L[1] *
           ((int64_t)c[2] + (int64_t)L[2] * (int64_t)c[3]));
}

static void lex_coords(const int32_t L[4], int64_t n, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) { c[mu] = (int)(n % L[mu]); n /= L[mu]; }
}

/* neighbour n +/- mu-hat with periodic wrap */
static int64_t neighbour(const int32_t L[4], const int c[4], int mu, int step)
{
    int d[4] = {c[0], c[1], c[2], c[3]};
    d[mu] = (d[mu] + step + L[mu]) % L[mu];
    return lex_index(L, d);
}

int64_t lq_oracle_volume(const int32_t L[4])
{
    return (int64_t)L[0] * L[1] * L[2] * L[3];
}

/* ------------------------------------------------------------------------------------
 * Eq. (1) for one output site n:
 *   (D psi)(n) = (m_q + 4) psi(n)
 *              + 1/2 sum_mu [ U_mu(n) P^{-mu} psi(n+mu) + U_mu(n-mu)^dag P^{+mu} psi(n-mu) ]
 * dagger != 0 gives D^dag, which is the same expression with P^{-mu} and P^{+mu}
 * exchanged (the transpose of the hopping term moves each link to the other side and
 * the Hermitian projectors are unchanged, so only the pairing of projector and hop
 * direction flips).
 * The product (P (x) U) psi is taken as U (P psi): first the 4x4 spin matrix on each
 * colour, then the 3x3 colour matrix on each spin.
 * ---------------------------------------------------------------------------------- */
static void site_apply(const int32_t L[4], double m_q, const cplx *U, const cplx *psi,
                       int64_t n, int dagger, cplx P[4][2][4][4], cplx out[4][3])
{
    int c[4];
    lex_coords(L, n, c);
    const cplx *pn = psi + 12 * n;
    for (int a = 0; a < 4; ++a)
        for (int A = 0; A < 3; ++A) out[a][A] = (m_q + 4.0) * pn[3 * a + A];

    for (int mu = 0; mu < 4; ++mu) {
        const int64_t nf = neighbour(L, c, mu, +1);
        const int64_t nb = neighbour(L, c, mu, -1);
        const cplx *Uf = U + 9 * (4 * n + mu);    /* U_mu(n)        */
        const cplx *Ub = U + 9 * (4 * nb + mu);   /* U_mu(n - mu)   */
        const cplx *pf = psi + 12 * nf;
        const cplx *pb = psi + 12 * nb;
        /* index 0 of P[mu][.] holds P^{-mu} = 1 - gamma, index 1 holds P^{+mu} = 1 + gamma */
        cplx (*Pf)[4] = P[mu][dagger ? 1 : 0];
        cplx (*Pb)[4] = P[mu][dagger ? 0 : 1];

        /* spin matrix on the neighbour spinors */
        cplx hf[4][3], hb[4][3];
        for (int a = 0; a < 4; ++a)
            for (int B = 0; B < 3; ++B) {
                cplx sf = 0.0, sb = 0.0;
                for (int b = 0; b < 4; ++b) {
                    sf += Pf[a][b] * pf[3 * b + B];
                    sb += Pb[a][b] * pb[3 * b + B];
                }
                hf[a][B] = sf;
                hb[a][B] = sb;
            }
        /* colour matrix: U_mu(n)^{AB} and (U_mu(n-mu)^dag)^{AB} = conj(U_mu(n-mu)^{BA}) */
        for (int a = 0; a < 4; ++a)
            for (int A = 0; A < 3; ++A) {
                cplx s = 0.0;
                for (int B = 0; B < 3; ++B) {
                    s += Uf[3 * A + B] * hf[a][B];
                    s += conj(Ub[3 * B + A]) * hb[a][B];
                }
                out[a][A] += 0.5 * s;
            }
    }
}

static void all_projectors(cplx P[4][2][4][4])
{
    for (int mu = 0; mu < 4; ++mu) {
        projector(mu, -1, P[mu][0]);
        projector(mu, +1, P[mu][1]);
    }
}

/* out = D psi (dagger = 0) or D^dag psi (dagger = 1) on the whole lattice.
 * out must not alias psi. */
void lq_oracle_dslash(const int32_t L[4], double m_q, const double *U_reals,
                      const double *psi_reals, double *out_reals, int dagger)
{
    cplx P[4][2][4][4];
    all_projectors(P);
    const int64_t V = lq_oracle_volume(L);
    const cplx *U = (const cplx *)U_reals;
    const cplx *psi = (const cplx *)psi_reals;
    cplx *out = (cplx *)out_reals;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
#endif
    for (int64_t n = 0; n < V; ++n) {
        cplx o[4][3];
        site_apply(L, m_q, U, psi, n, dagger, P, o);
        for (int a = 0; a < 4; ++a)
            for (int A = 0; A < 3; ++A) out[12 * n + 3 * a + A] = o[a][A];
    }
}

/* Eq. (1) at a list of sites only: out[k] = (D psi)(sites[k]); used to check full-size
 * results on a sample of output sites. */
void lq_oracle_dslash_sites(const int32_t L[4], double m_q, const double *U_reals,
                            const double *psi_reals, int64_t nsites, const int64_t *sites,
                            double *out_reals, int dagger)
{
    cplx P[4][2][4][4];
    all_projectors(P);
    const cplx *U = (const cplx *)U_reals;
    const cplx *psi = (const cplx *)psi_reals;
    cplx *out = (cplx *)out_reals;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) num_threads(g_threads) if (g_threads > 1)
#endif
    for (int64_t k = 0; k < nsites; ++k) {
        cplx o[4][3];
        site_apply(L, m_q, U, psi, sites[k], dagger, P, o);
        for (int a = 0; a < 4; ++a)
            for (int A = 0; A < 3; ++A) out[12 * k + 3 * a + A] = o[a][A];
    }
}

/* ------------------------------------------------------------------------------------
 * Vector helpers for the solvers (length 12 V complex).
 * <a, b> = sum conj(a) b over all sites, spins, colours.
 * ---------------------------------------------------------------------------------- */
static cplx vdot(int64_t n, const cplx *a, const cplx *b)
{
    cplx s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += conj(a[i]) * b[i];
    return s;
}

static double vnorm2(int64_t n, const cplx *a)
{
    return creal(vdot(n, a, a));
}

/* A = D^dag D applied as two operator calls through a temporary. */
static void normal_op(const int32_t L[4], double m_q, const double *U, const cplx *in,
                      cplx *tmp, cplx *out)
{
    lq_oracle_dslash(L, m_q, U, (const double *)in, (double *)tmp, 0);
    lq_oracle_dslash(L, m_q, U, (const double *)tmp, (double *)out, 1);
}

void lq_oracle_normal_op(const int32_t L[4], double m_q, const double *U_reals,
                         const double *in_reals, double *out_reals)
{
    const int64_t n = 12 * lq_oracle_volume(L);
    cplx *tmp = (cplx *)malloc(sizeof(cplx) * n);
    normal_op(L, m_q, U_reals, (const cplx *)in_reals, tmp, (cplx *)out_reals);
    free(tmp);
}

/* ------------------------------------------------------------------------------------
 * Textbook conjugate gradient (Hestenes-Stiefel) on A = D^dag D, FP64.
 * Solves A x = eta starting from the x passed in.  Stops when the iterated residual
 * satisfies ||r|| <= tol ||eta|| or after max_iter iterations; then recomputes the true
 * residual ||eta - A x|| / ||eta||.  Returns 0 if that true residual is <= tol, 1 if not.
 * ---------------------------------------------------------------------------------- */
int lq_oracle_cg(const int32_t L[4], double m_q, const double *U_reals,
                 const double *eta_reals, double *x_reals, double tol, int32_t max_iter,
                 int32_t *iters_out, double *true_rel_out)
{
    const int64_t n = 12 * lq_oracle_volume(L);
    const cplx *eta = (const cplx *)eta_reals;
    cplx *x = (cplx *)x_reals;
    cplx *r = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *q = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n);

    normal_op(L, m_q, U_reals, x, tmp, q);
    for (int64_t i = 0; i < n; ++i) { r[i] = eta[i] - q[i]; p[i] = r[i]; }
    const double eta2 = vnorm2(n, eta);
    double rr = vnorm2(n, r);
    int k = 0;
    while (k < max_iter && sqrt(rr) > tol * sqrt(eta2)) {
        normal_op(L, m_q, U_reals, p, tmp, q);
        const double alpha = rr / creal(vdot(n, p, q));
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        const double rr_new = vnorm2(n, r);
        const double beta = rr_new / rr;
        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
        ++k;
    }
    normal_op(L, m_q, U_reals, x, tmp, q);
    for (int64_t i = 0; i < n; ++i) r[i] = eta[i] - q[i];
    const double true_rel = sqrt(vnorm2(n, r) / eta2);
    if (iters_out) *iters_out = k;
    if (true_rel_out) *true_rel_out = true_rel;
    free(r); free(p); free(q); free(tmp);
    return true_rel <= tol ? 0 : 1;
}

/* ------------------------------------------------------------------------------------
 * Algorithm 1 (residual-guided mixed-precision CG), taken step by step in the paper's
 * order.  "High" quantities are FP64.  "Low" quantities are FP64 numbers rounded to
 * FP32 after every vector operation when low_is_f32 != 0 (and left in FP64 otherwise);
 * the low operator is the FP64 operator applied to the rounded vector, rounded again.
 *
 * Readings of the algorithm's open points:
 *   - eta (first residual) and b (later residuals) are the same right-hand side;
 *   - at the start of cycle l, r_0 = r^high_l / s^high_l (the text's l+1 index is
 *     read as the residual computed at the end of the previous cycle);
 *   - search direction: in the first cycle p_0 = r_0; afterwards
 *       p_0 = r_0 + beta_0 (p_k - <r_0, p_k> r_0),   beta_0 = s_l / (s_{l-1} rho_k),
 *     i.e. the old direction, with its component along the new residual removed, is
 *     continued with the CG coefficient rescaled into the unit-norm units of r_0;
 *   - that continuation is exact only while the inner recurrence tracks the true
 *     residual, s_l = s_{l-1} sqrt(rho_k) up to rounding.  When the new true residual
 *     exceeds twice the recurrence's prediction (s_l > 2 s_{l-1} sqrt(rho_k): once the
 *     tolerance lies below what the high precision resolves, the residual is rounding noise
 *     and beta_0 ~ 1/rho_k would blow the stale direction up), the cycle starts afresh
 *     from p_0 = r_0, as the first one does;
 *   - rho_0 = ||r_0||^2 (one, up to the rounding of r_0);
 *   - the solution update is psi^high += s_l psi_k, where psi_k already holds all k
 *     inner updates;
 *   - the inner loop runs while n < k_max and rho_n > max(delta^2, (tol ||eta|| / s_l)^2);
 *   - the outer loop runs while s^high > tol ||eta|| (relative stopping criterion).
 * Returns 0 if the final true residual is <= tol, 1 otherwise.
 * ---------------------------------------------------------------------------------- */
static void round_low(int64_t n, cplx *v, int low_is_f32)
{
    if (!low_is_f32) return;
    for (int64_t i = 0; i < n; ++i)
        v[i] = (double)(float)creal(v[i]) + I * (double)(float)cimag(v[i]);
}

int lq_oracle_alg1(const int32_t L[4], double m_q, const double *U_reals,
                   const double *eta_reals, double *x_reals, double tol, int low_is_f32,
                   double delta, int32_t k_max, int32_t max_cycles,
                   int32_t *cycles_out, int32_t *inner_total_out, double *true_rel_out)
{
    const int64_t n = 12 * lq_oracle_volume(L);
    const cplx *eta = (const cplx *)eta_reals;
    cplx *x_high = (cplx *)x_reals;                       /* psi^high          */
    cplx *r_high = malloc(sizeof(cplx) * n);
    cplx *tmp = malloc(sizeof(cplx) * n), *q = malloc(sizeof(cplx) * n);
    cplx *psi = malloc(sizeof(cplx) * n), *r = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n);

    const double eta_norm = sqrt(vnorm2(n, eta));
    /* r_0^high = eta - (D^dag D)^high psi^high ; s_0^high = ||r_0^high|| */
    normal_op(L, m_q, U_reals, x_high, tmp, q);
    for (int64_t i = 0; i < n; ++i) r_high[i] = eta[i] - q[i];
    double s = sqrt(vnorm2(n, r_high)), s_prev = 0.0, rho = 1.0;
    int l = 0, inner_total = 0, fresh = 1;

    while (s > tol * eta_norm && l < max_cycles) {
        /* psi_0 = 0 ; r_0 = r^high / s^high */
        for (int64_t i = 0; i < n; ++i) { psi[i] = 0.0; r[i] = r_high[i] / s; }
        round_low(n, r, low_is_f32);
        if (fresh) {
            for (int64_t i = 0; i < n; ++i) p[i] = r[i];
        } else {
            /* p_0 = r_0 + beta_0 (p_k - <r_0, p_k> r_0),  beta_0 = s_l / (s_{l-1} rho_k) */
            const double beta0 = s / (s_prev * rho);
            const cplx c = vdot(n, r, p);
            for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta0 * (p[i] - c * r[i]);
        }
        round_low(n, p, low_is_f32);
        rho = vnorm2(n, r);
        const double target = tol * eta_norm / s;
        const double stop = fmax(delta * delta, target * target);
        int k = 0;
        while (k < k_max && rho > stop) {
            /* q_n = D^dag D p_n (low) */
            normal_op(L, m_q, U_reals, p, tmp, q);
            round_low(n, q, low_is_f32);
            const double alpha = rho / creal(vdot(n, p, q));
            for (int64_t i = 0; i < n; ++i) { psi[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
            round_low(n, psi, low_is_f32);
            round_low(n, r, low_is_f32);
            const double rho_new = vnorm2(n, r);
            const double beta = rho_new / rho;
            for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
            round_low(n, p, low_is_f32);
            rho = rho_new;
            ++k;
        }
        inner_total += k;
        /* psi^high_{l+1} = psi^high_l + s_l psi_k */
        for (int64_t i = 0; i < n; ++i) x_high[i] += s * psi[i];
        /* r^high_{l+1} = b - (D^dag D)^high psi^high_{l+1} ; s_{l+1} = ||r^high_{l+1}|| */
        normal_op(L, m_q, U_reals, x_high, tmp, q);
        for (int64_t i = 0; i < n; ++i) r_high[i] = eta[i] - q[i];
        const double s_new = sqrt(vnorm2(n, r_high));
        fresh = !(s_new <= 2.0 * s * sqrt(rho));
        s_prev = s;
        s = s_new;
        ++l;
        if (k == 0) break;   /* no progress possible */
    }
    const double true_rel = s / eta_norm;
    if (cycles_out) *cycles_out = l;
    if (inner_total_out) *inner_total_out = inner_total;
    if (true_rel_out) *true_rel_out = true_rel;
    free(r_high); free(tmp); free(q); free(psi); free(r); free(p);
    return true_rel <= tol ? 0 : 1;
}

/* ------------------------------------------------------------------------------------
 * 12-real link format: rows 0 and 1 are stored; for an SU(3) matrix the third row is
 * the complex conjugate of the cross product of the first two,
 *   u2 = conj(u0 x u1),  (a x b)_i = eps_ijk a_j b_k,
 * because U^{-1} = U^dag = adj(U) when det U = 1.
 * in: [nlinks][2][3] complex, out: [nlinks][3][3] complex.
 * ---------------------------------------------------------------------------------- */
void lq_oracle_reconstruct12(int64_t nlinks, const double *rows_reals, double *full_reals)
{
    const cplx *in = (const cplx *)rows_reals;
    cplx *out = (cplx *)full_reals;
    for (int64_t k = 0; k < nlinks; ++k) {
        const cplx *a = in + 6 * k, *b = in + 6 * k + 3;
        cplx *o = out + 9 * k;
        for (int j = 0; j < 3; ++j) { o[j] = a[j]; o[3 + j] = b[j]; }
        o[6] = conj(a[1] * b[2] - a[2] * b[1]);
        o[7] = conj(a[2] * b[0] - a[0] * b[2]);
        o[8] = conj(a[0] * b[1] - a[1] * b[0]);
    }
}

/* ------------------------------------------------------------------------------------
 * 10-real link format.  The paper streams each link as 10 input words instead of 18
 * (Introduction; Section 2.2), chosen so that no trigonometric function is needed, but the
 * construction it cites is not in the text.  This one follows from unitarity alone:
 *   stored: row 0 (u00, u01, u02) and the two entries of row 1 outside column k, in
 *     increasing column order, where k is the column of row 0 whose larger component
 *     max(|Re u0k|, |Im u0k|) is the largest (the lowest such column on ties), decided on
 *     the stored values;
 *   rebuilt: rows 0 and 1 of a unitary matrix are orthogonal, sum_j u1j conj(u0j) = 0, so
 *       u1k = -(sum_{j != k} u1j conj(u0j)) / conj(u0k),
 *     and row 2 = conj(row0 x row1) as in the 12-real form.
 * Row 0 has unit norm, so some column has |u0j|^2 >= 1/3, hence a component of magnitude
 * >= 1/sqrt(6); the chosen column therefore has |u0k| >= 1/sqrt(6), which bounds the
 * amplification of the stored values' rounding by the division.
 * in: [nlinks][5] complex, out: [nlinks][3][3] complex.
 * ---------------------------------------------------------------------------------- */
static double larger_part(cplx z)
{
    const double a = fabs(creal(z)), b = fabs(cimag(z));
    return a > b ? a : b;
}

void lq_oracle_reconstruct10(int64_t nlinks, const double *stored_reals, double *full_reals)
{
    const cplx *in = (const cplx *)stored_reals;
    cplx *out = (cplx *)full_reals;
    for (int64_t n = 0; n < nlinks; ++n) {
        const cplx *w = in + 5 * n;
        cplx *o = out + 9 * n;
        int k = 0;
        for (int j = 1; j < 3; ++j)
            if (larger_part(w[j]) > larger_part(w[k])) k = j;
        for (int j = 0; j < 3; ++j) o[j] = w[j];
        /* row 1: the stored entries fill the columns other than k, in increasing order */
        int at = 3;
        cplx sum = 0.0;
        for (int j = 0; j < 3; ++j) {
            if (j == k) continue;
            o[3 + j] = w[at++];
            sum += o[3 + j] * conj(w[j]);
        }
        o[3 + k] = -sum / conj(w[k]);
        const cplx *a = o, *b = o + 3;
        o[6] = conj(a[1] * b[2] - a[2] * b[1]);
        o[7] = conj(a[2] * b[0] - a[0] * b[2]);
        o[8] = conj(a[0] * b[1] - a[1] * b[0]);
    }
}
