/*
 * rbsog_oracle.c -- plain FP64 CPU oracle of the RBSOG electrostatics path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA path (paper_2602_23582_gb300/).
 *
 * Every function follows a passage of arXiv 2602.23582 ("Random batch
 * sum-of-Gaussians method for molecular dynamics simulation of particle
 * systems in the NPT ensemble"), cited by section / equation label:
 *
 *   orc_sog_terms        sec. 2.2 (w_l, s_l of eq. long) and sec. 3.1
 *                        (w~_l, s~_l; eq. omega0: omega rescales l = 0)
 *   orc_sog_solve        eqs. Eq::2.20 / eq::2.22 (C0 and C1 at r_c)
 *   orc_bsa              eq. BSA_beta (bilateral series), bound eq. BSA_err
 *   orc_short_range      eqs. U_short, force_SOG, P_short (direct sums)
 *   orc_kspace_all       eqs. U_long, force_SOG (Fourier part), P_long
 *   orc_pf_realspace     eq. PFcoul (real-space image sum of P^F)
 *   orc_normalizers      eqs. Sr, Snr (lattice sums H^r_l, H^nr_l)
 *   orc_normalizers_3d   the same lattice sums, summed over Z^3 directly
 *   orc_normalizers_poisson  Proposition 3.5 (eqs. H2, H2r)
 *   orc_sample_modes     App. D (MH for P^r, eqs. proposal, acc_Gaussian)
 *                        and sec. 3.2 (measure-recalibration chain)
 *   orc_distinct         sec. 3.2 (distinct modes of the union)
 *   orc_rho              eq. rho_k
 *   orc_rb_longrange     eqs. P_approx_r, P_approx_nr, f_approx (App. B),
 *                        U_long estimated with the same radial samples
 *   orc_nr_shared        sec. 3.2: the shared-proposal (non-recalibrated)
 *                        estimator of eq. PcoulFnr from the radial samples
 *   orc_self_energy      App. A (U_self)
 *   orc_exclusions       intramolecular pairs removed from the Fourier part
 *   orc_bonded           harmonic bonds and angles
 *   orc_force_eval       Algorithm 1 steps 2-7 for one configuration
 *   orc_npt_run          Algorithm 1 step 8 with eq. Langevin_NPT
 *   orc_tri_*, orc_rho_h, orc_rb_longrange_h, orc_force_eval_h, orc_nvt_run_h
 *                        the same steps for a general (triclinic) cell h:
 *                        k = 2 pi h^{-T} m (eq. Sr), eq. proposal as a
 *                        Gaussian integral over the cube around m*, lattice
 *                        sums over Z^3 (eqs. Sr, Snr)
 *
 * Conventions shared with the inputs (not with the CUDA code): LAMMPS "real"
 * units; h is row-major with the cell vectors as its columns (r = h s);
 * positions are N x 3 row-major.  The paper writes Coulomb in Gaussian units,
 * so every Coulomb energy, force and virial carries the factor ke.
 *
 * Parity status: every function above is pinned by a CPU test against a
 * value the paper prints, a closed form, an independent identity or a brute
 * force evaluation (tests/test_oracle_*.py).  Compile with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

static int orc_team_size(void)
{
#ifdef _OPENMP
    return omp_get_num_threads();
#else
    return 1;
#endif
}
#define ORC_MAXM 256

/* ------------------------------------------------------------------------ */
/* SOG parameters                                                            */
/* ------------------------------------------------------------------------ */

/* sec. 2.2: w_l = (pi/2)^{-1/2} sigma^{-1} b^{-l} log b, s_l = sqrt(2) b^l sigma;
 * sec. 3.1: w~_l = (pi/2)^{-1/2} log b / (b^{3l} sigma^3), s~_l = s_l (b~ = b,
 * sigma~ = sigma); eq. omega0 and its energy analogue: both l = 0 weights are
 * multiplied by omega. */
void orc_sog_terms(double b, double sigma, double omega, int M,
                   double *w, double *s, double *wt, double *st)
{
    const double c = sqrt(2.0 / ORC_PI);
    const double lb = log(b);
    for (int l = 0; l < M; ++l) {
        double bl = pow(b, (double)l);
        s[l] = sqrt(2.0) * bl * sigma;
        st[l] = s[l];
        w[l] = c * lb / (sigma * bl);
        wt[l] = c * lb / (bl * bl * bl * sigma * sigma * sigma);
    }
    w[0] *= omega;
    wt[0] *= omega;
}

/* 1/r - F(r) and its C1 partner r^3 F~(r) - 1 evaluated at x = r_c / sigma
 * with the Gaussian series untruncated above (l = 0 .. inf): with omega
 * eliminated through the C0 condition, the C1 residual is
 * h(x) = (1 - B1(x)) x^2 + B2(x) - 1. */
static void sog_solve_parts(double b, double x, double *A1, double *B1,
                            double *B2, double *dB1, double *dB2)
{
    const double c = sqrt(2.0 / ORC_PI), lb = log(b);
    int L = (int)ceil(46.0 / lb);
    double b1 = 0, b2 = 0, d1 = 0, d2 = 0;
    for (int l = 1; l < L; ++l) {
        double bl = pow(b, (double)l);
        double e = exp(-x * x / (2.0 * bl * bl));
        b1 += c * lb * x / bl * e;
        b2 += c * lb * x * x * x / (bl * bl * bl) * e;
        d1 += c * lb / bl * e * (1.0 - x * x / (bl * bl));
        d2 += c * lb / (bl * bl * bl) * e * (3.0 * x * x - x * x * x * x / (bl * bl));
    }
    *A1 = c * x * lb * exp(-x * x / 2.0);
    *B1 = b1; *B2 = b2; *dB1 = d1; *dB2 = d2;
}

static double sog_h(double b, double x)
{
    double A1, B1, B2, d1, d2;
    sog_solve_parts(b, x, &A1, &B1, &B2, &d1, &d2);
    return (1.0 - B1) * x * x + B2 - 1.0;
}

static double sog_hp(double b, double x)
{
    double A1, B1, B2, d1, d2;
    sog_solve_parts(b, x, &A1, &B1, &B2, &d1, &d2);
    return -d1 * x * x + 2.0 * x * (1.0 - B1) + d2;
}

/* Given (b, r_c), find (sigma, omega) making 1/r - F and 1/r^3 - F~ vanish at
 * r_c (eqs. Eq::2.20, eq::2.22 / eq::continuity; with w_l = w~_l s~_l^2 / 2 the
 * second is the C1 condition, App. C).  The scan runs over x = r_c / sigma
 * upward and takes the first solution: a sign change of h, or a local
 * maximum of h that touches zero (a double root, which is how rows 2-4 of
 * Table 2 sit).  Returns 0 on success and the residuals in resid[2]. */
int orc_sog_solve(double b, double rc, double *sigma, double *omega, double *resid)
{
    const double dx = 0.005;
    double xprev = 0.5, hprev = sog_h(b, xprev), hpprev = sog_hp(b, xprev);
    for (double x = xprev + dx; x < 12.0; x += dx) {
        double hx = sog_h(b, x), hpx = sog_hp(b, x);
        double root = -1.0;
        if (hprev == 0.0) {
            root = xprev;
        } else if ((hprev < 0) != (hx < 0)) {
            double lo = xprev, hi = x, flo = hprev;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi), fm = sog_h(b, mid);
                if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
            }
            root = 0.5 * (lo + hi);
            /* rounding can make a double root look like a sign change: prefer
             * the extremum of h nearby when it touches zero */
            double a0 = xprev - dx, a1 = x + dx;
            if (sog_hp(b, a0) > 0 && sog_hp(b, a1) <= 0) {
                for (int it = 0; it < 200; ++it) {
                    double mid = 0.5 * (a0 + a1);
                    if (sog_hp(b, mid) > 0) a0 = mid; else a1 = mid;
                }
                double xm = 0.5 * (a0 + a1);
                if (fabs(sog_h(b, xm)) < 1e-12) root = xm;
            }
        } else if (hpprev > 0 && hpx <= 0) {
            double lo = xprev, hi = x;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (sog_hp(b, mid) > 0) lo = mid; else hi = mid;
            }
            double xm = 0.5 * (lo + hi);
            if (fabs(sog_h(b, xm)) < 1e-12) root = xm;
        }
        if (root > 0) {
            double A1, B1, B2, d1, d2;
            sog_solve_parts(b, root, &A1, &B1, &B2, &d1, &d2);
            *sigma = rc / root;
            *omega = (1.0 - B1) / A1;
            resid[0] = *omega * A1 + B1 - 1.0;
            resid[1] = sog_h(b, root);
            return 0;
        }
        xprev = x; hprev = hx; hpprev = hpx;
    }
    return -1;
}

/* eq. BSA_beta: 2 log b / ((sqrt2 sigma)^beta Gamma(beta/2)) *
 * sum_{l=lmin}^{lmax} b^{-beta l} exp(-(r / (b^l sigma))^2 / 2). */
double orc_bsa(double beta, double b, double sigma, double r, int lmin, int lmax)
{
    double sum = 0.0;
    for (int l = lmin; l <= lmax; ++l) {
        double bl = pow(b, (double)l);
        double t = r / (bl * sigma);
        sum += pow(b, -beta * l) * exp(-0.5 * t * t);
    }
    return 2.0 * log(b) / (pow(sqrt(2.0) * sigma, beta) * tgamma(0.5 * beta)) * sum;
}

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its        */
/* published definition.  The paper does not name its random generator.      */
/* ------------------------------------------------------------------------ */

void orc_philox(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * x0;
        unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ULL * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0, y1 = lo1, y2 = hi0 ^ x3 ^ k1, y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B97F4A7C15ULL;
        k1 += 0xBB67AE8584CAA73BULL;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* uniform in the open interval (0,1): ((x >> 12) + 1/2) 2^-52, exact in FP64
 * (the 53-bit analogue would round its top value to 1). */
double orc_u01(uint64_t x) { return ((double)(x >> 12) + 0.5) * (1.0 / 4503599627370496.0); }

static void draw4(uint64_t seed, uint64_t sysid, uint64_t step, uint64_t purpose,
                  uint64_t index, uint64_t out[4])
{
    uint64_t ctr[4] = {step, purpose, index, 0};
    uint64_t key[2] = {seed, sysid};
    orc_philox(ctr, key, out);
}

/* Box-Muller: (sqrt(-2 log u1) cos(2 pi u2), sqrt(-2 log u1) sin(2 pi u2)). */
static void box_muller(uint64_t a, uint64_t b, double *z0, double *z1)
{
    double u1 = orc_u01(a), u2 = orc_u01(b);
    double rr = sqrt(-2.0 * log(u1));
    double ang = 2.0 * ORC_PI * u2;
    *z0 = rr * cos(ang);
    *z1 = rr * sin(ang);
}

/* ------------------------------------------------------------------------ */
/* small linear algebra for a general cell h                                 */
/* ------------------------------------------------------------------------ */

static double det3(const double *h)
{
    return h[0] * (h[4] * h[8] - h[5] * h[7]) - h[1] * (h[3] * h[8] - h[5] * h[6])
         + h[2] * (h[3] * h[7] - h[4] * h[6]);
}

static void inv3(const double *h, double *hi)
{
    double d = det3(h);
    hi[0] = (h[4] * h[8] - h[5] * h[7]) / d;
    hi[1] = (h[2] * h[7] - h[1] * h[8]) / d;
    hi[2] = (h[1] * h[5] - h[2] * h[4]) / d;
    hi[3] = (h[5] * h[6] - h[3] * h[8]) / d;
    hi[4] = (h[0] * h[8] - h[2] * h[6]) / d;
    hi[5] = (h[2] * h[3] - h[0] * h[5]) / d;
    hi[6] = (h[3] * h[7] - h[4] * h[6]) / d;
    hi[7] = (h[1] * h[6] - h[0] * h[7]) / d;
    hi[8] = (h[0] * h[4] - h[1] * h[3]) / d;
}

/* minimum image of d through fractional coordinates: d <- h (s - rint(s)) */
static void min_image(const double *h, const double *hi, double *d)
{
    double s[3];
    for (int a = 0; a < 3; ++a) {
        s[a] = hi[3 * a] * d[0] + hi[3 * a + 1] * d[1] + hi[3 * a + 2] * d[2];
        s[a] -= nearbyint(s[a]);
    }
    for (int a = 0; a < 3; ++a) d[a] = h[3 * a] * s[0] + h[3 * a + 1] * s[1] + h[3 * a + 2] * s[2];
}

static void diag_box(const double L[3], double *h)
{
    memset(h, 0, 9 * sizeof(double));
    h[0] = L[0]; h[4] = L[1]; h[8] = L[2];
}

/* ------------------------------------------------------------------------ */
/* cell binning (used only to compare membership sets with the CUDA path)    */
/* ------------------------------------------------------------------------ */

/* s = r / L wrapped into [0,1) (1.0 mapped to 0), n = floor(L * sub / r_c) cells
 * per axis, cell = min(floor(s n), n - 1), cell index x fastest. */
void orc_cell_bin(int N, const double *r, const double L[3], double rc, int sub,
                  int *ncell, int *cell)
{
    for (int a = 0; a < 3; ++a) ncell[a] = (int)floor(L[a] * sub / rc);
    for (int i = 0; i < N; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double s = r[3 * i + a] / L[a];
            s = s - floor(s);
            if (s >= 1.0) s = 0.0;
            int k = (int)floor(s * ncell[a]);
            if (k > ncell[a] - 1) k = ncell[a] - 1;
            c[a] = k;
        }
        cell[i] = c[0] + ncell[0] * (c[1] + ncell[1] * c[2]);
    }
}

/* ------------------------------------------------------------------------ */
/* short-range part: direct sums over all pairs, minimum image               */
/* ------------------------------------------------------------------------ */

/* eqs. U_short, force_SOG (short-range force, kernel N~ = 1/r^3 - F~) and
 * P_short (virial f (x) r), all pairs with r < r_c and different molecule ids;
 * plus a 12-6 Lennard-Jones term cut (not shifted) at r_c.  F is accumulated
 * (+=).  en[0] = U^N_coul, en[1] = U_LJ; Wc, Wl = Coulomb and LJ virials
 * (kcal/mol). */
void orc_short_range(int N, const double *r, const double *q, const int *type,
                     const int *mol, const double *h, double rc,
                     int M, const double *wt, const double *st,
                     int ME, const double *w, const double *s,
                     int ntypes, const double *lj_eps, const double *lj_sig,
                     double ke, double *F, double *en, double *Wc, double *Wl)
{
    double hi[9];
    inv3(h, hi);
    const double rc2 = rc * rc;
    double Uc = 0, Ul = 0, wc[9] = {0}, wl[9] = {0};
#pragma omp parallel
    {
        double uc = 0, ul = 0, tc[9] = {0}, tl[9] = {0};
#pragma omp for schedule(static)
        for (int i = 0; i < N; ++i) {
            double fi[3] = {0, 0, 0};
            for (int j = 0; j < N; ++j) {
                if (j == i || mol[i] == mol[j]) continue;
                double d[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
                min_image(h, hi, d);
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 >= rc2) continue;
                double rr = sqrt(r2);
                double fs = 1.0 / (r2 * rr), es = 1.0 / rr;
                for (int l = 0; l < M; ++l) fs -= wt[l] * exp(-r2 / (st[l] * st[l]));
                for (int l = 0; l < ME; ++l) es -= w[l] * exp(-r2 / (s[l] * s[l]));
                double qq = ke * q[i] * q[j];
                double f = qq * fs;
                uc += 0.5 * qq * es;
                double eps = lj_eps[type[i] * ntypes + type[j]];
                double fl = 0.0;
                if (eps != 0.0) {
                    double sg = lj_sig[type[i] * ntypes + type[j]];
                    double sr2 = sg * sg / r2, sr6 = sr2 * sr2 * sr2;
                    ul += 0.5 * 4.0 * eps * (sr6 * sr6 - sr6);
                    fl = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
                }
                for (int a = 0; a < 3; ++a) {
                    fi[a] += (f + fl) * d[a];
                    for (int b = 0; b < 3; ++b) {
                        tc[3 * a + b] += 0.5 * f * d[a] * d[b];
                        tl[3 * a + b] += 0.5 * fl * d[a] * d[b];
                    }
                }
            }
            for (int a = 0; a < 3; ++a) F[3 * i + a] += fi[a];
        }
#pragma omp for ordered schedule(static, 1)
        for (int t = 0; t < orc_team_size(); ++t) {
#pragma omp ordered
            {
                Uc += uc; Ul += ul;
                for (int a = 0; a < 9; ++a) { wc[a] += tc[a]; wl[a] += tl[a]; }
            }
        }
    }
    en[0] = Uc; en[1] = Ul;
    for (int a = 0; a < 9; ++a) { Wc[a] = wc[a]; Wl[a] = wl[a]; }
}

/* The same sums over cell lists (used by the timed CPU baseline only): for
 * an orthorhombic h with at least 3 cells of >= r_c per axis, every pair
 * within r_c lies in the 27 cells around i's cell.  The hits of atom i are
 * gathered from those cells with the same minimum-image arithmetic as above,
 * sorted by j, and then evaluated and added in ascending j exactly as the
 * all-pairs loop adds them (same expressions, same order, same static split
 * of i over the threads), so the results are bit for bit those of
 * orc_short_range.  Returns -1 (nothing computed) when h is not diagonal or
 * a box edge holds fewer than 3 cells. */
typedef struct { int j; double d[3]; double r2; } orc_hit;

static int cmp_hit(const void *a, const void *b)
{
    const int x = ((const orc_hit *)a)->j, y = ((const orc_hit *)b)->j;
    return (x > y) - (x < y);
}

int orc_short_range_cells(int N, const double *r, const double *q, const int *type,
                          const int *mol, const double *h, double rc,
                          int M, const double *wt, const double *st,
                          int ME, const double *w, const double *s,
                          int ntypes, const double *lj_eps, const double *lj_sig,
                          double ke, double *F, double *en, double *Wc, double *Wl)
{
    if (h[1] != 0 || h[2] != 0 || h[3] != 0 || h[5] != 0 || h[6] != 0 || h[7] != 0) return -1;
    const double L[3] = {h[0], h[4], h[8]};
    int nc[3];
    for (int a = 0; a < 3; ++a) {
        nc[a] = (int)floor(L[a] / rc);
        if (nc[a] < 3) return -1;
    }
    const int C = nc[0] * nc[1] * nc[2];
    int *cell = (int *)malloc(sizeof(int) * (size_t)N);
    int *start = (int *)calloc((size_t)C + 1, sizeof(int));
    int *list = (int *)malloc(sizeof(int) * (size_t)N);
    for (int i = 0; i < N; ++i) {
        int c[3];
        for (int a = 0; a < 3; ++a) {
            double u = r[3 * i + a] / L[a];
            u = u - floor(u);
            if (u >= 1.0) u = 0.0;
            int k = (int)floor(u * nc[a]);
            if (k > nc[a] - 1) k = nc[a] - 1;
            if (k < 0) k = 0;
            c[a] = k;
        }
        cell[i] = c[0] + nc[0] * (c[1] + nc[1] * c[2]);
        ++start[cell[i] + 1];
    }
    for (int c = 0; c < C; ++c) start[c + 1] += start[c];
    {
        int *fill = (int *)malloc(sizeof(int) * (size_t)C);
        memcpy(fill, start, sizeof(int) * (size_t)C);
        for (int i = 0; i < N; ++i) list[fill[cell[i]]++] = i;   /* ascending index within a cell */
        free(fill);
    }
    double hi[9];
    inv3(h, hi);
    const double rc2 = rc * rc;
    double Uc = 0, Ul = 0, wc[9] = {0}, wl[9] = {0};
#pragma omp parallel
    {
        double uc = 0, ul = 0, tc[9] = {0}, tl[9] = {0};
        int cap = 1024;
        orc_hit *hits = (orc_hit *)malloc(sizeof(orc_hit) * (size_t)cap);
#pragma omp for schedule(static)
        for (int i = 0; i < N; ++i) {
            const int ci = cell[i];
            const int cx = ci % nc[0], cy = (ci / nc[0]) % nc[1], cz = ci / (nc[0] * nc[1]);
            int nh = 0;
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int g = (cx + dx + nc[0]) % nc[0] +
                                      nc[0] * ((cy + dy + nc[1]) % nc[1] + nc[1] * ((cz + dz + nc[2]) % nc[2]));
                        for (int k = start[g]; k < start[g + 1]; ++k) {
                            const int j = list[k];
                            if (j == i || mol[i] == mol[j]) continue;
                            double d[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1],
                                           r[3 * i + 2] - r[3 * j + 2]};
                            min_image(h, hi, d);
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (r2 >= rc2) continue;
                            if (nh == cap) {
                                cap *= 2;
                                hits = (orc_hit *)realloc(hits, sizeof(orc_hit) * (size_t)cap);
                            }
                            hits[nh].j = j;
                            hits[nh].d[0] = d[0]; hits[nh].d[1] = d[1]; hits[nh].d[2] = d[2];
                            hits[nh].r2 = r2;
                            ++nh;
                        }
                    }
            qsort(hits, (size_t)nh, sizeof(orc_hit), cmp_hit);
            double fi[3] = {0, 0, 0};
            for (int e = 0; e < nh; ++e) {
                const int j = hits[e].j;
                const double *d = hits[e].d;
                const double r2 = hits[e].r2;
                double rr = sqrt(r2);
                double fs = 1.0 / (r2 * rr), es = 1.0 / rr;
                for (int l = 0; l < M; ++l) fs -= wt[l] * exp(-r2 / (st[l] * st[l]));
                for (int l = 0; l < ME; ++l) es -= w[l] * exp(-r2 / (s[l] * s[l]));
                double qq = ke * q[i] * q[j];
                double f = qq * fs;
                uc += 0.5 * qq * es;
                double eps = lj_eps[type[i] * ntypes + type[j]];
                double fl = 0.0;
                if (eps != 0.0) {
                    double sg = lj_sig[type[i] * ntypes + type[j]];
                    double sr2 = sg * sg / r2, sr6 = sr2 * sr2 * sr2;
                    ul += 0.5 * 4.0 * eps * (sr6 * sr6 - sr6);
                    fl = 24.0 * eps * (2.0 * sr6 * sr6 - sr6) / r2;
                }
                for (int a = 0; a < 3; ++a) {
                    fi[a] += (f + fl) * d[a];
                    for (int b = 0; b < 3; ++b) {
                        tc[3 * a + b] += 0.5 * f * d[a] * d[b];
                        tl[3 * a + b] += 0.5 * fl * d[a] * d[b];
                    }
                }
            }
            for (int a = 0; a < 3; ++a) F[3 * i + a] += fi[a];
        }
        free(hits);
#pragma omp for ordered schedule(static, 1)
        for (int t = 0; t < orc_team_size(); ++t) {
#pragma omp ordered
            {
                Uc += uc; Ul += ul;
                for (int a = 0; a < 9; ++a) { wc[a] += tc[a]; wl[a] += tl[a]; }
            }
        }
    }
    en[0] = Uc; en[1] = Ul;
    for (int a = 0; a < 9; ++a) { Wc[a] = wc[a]; Wl[a] = wl[a]; }
    free(cell); free(start); free(list);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* deterministic Fourier part over all modes                                */
/* ------------------------------------------------------------------------ */

/* For every m != 0 with |m_a| <= mmax[a]: k = 2 pi h^{-T} m, rho(k) (eq. rho_k),
 *   U^F   += (1/2V) Fhat_E(k) |rho|^2,  Fhat_E = sum_{l<ME} pi^1.5 w s^3 e^{-s^2k^2/4}
 *   F_i   += -(q_i/V) k Fhat_F(k) Im(e^{-ik.r_i} rho),
 *            Fhat_F = sum_{l<M} (pi^1.5/2) w~ s~^5 e^{-s~^2 k^2/4}
 *            (the Fourier transform of F for the consistent set w = w~ s~^2/2)
 *   P^F   += pi^1.5/(4V^2) sum_l w~ s~^5 e^{..} (I - s~^2/2 k (x) k) |rho|^2  (eq. P_long)
 * All times ke.  F is accumulated; UF[0] returned; WF[9] is the virial V P^F
 * in kcal/mol and WFr[0] (optional) its radial part (eq. PcoulFr). */
void orc_kspace_all(int N, const double *r, const double *q, const double *h,
                    int M, const double *wt, const double *st,
                    int ME, const double *w, const double *s,
                    const int *mmax, double ke, double *F, double *UF, double *WF,
                    double *WFr)
{
    double hi[9];
    inv3(h, hi);
    const double V = fabs(det3(h));
    const double pi15 = pow(ORC_PI, 1.5);
    int nx = 2 * mmax[0] + 1, ny = 2 * mmax[1] + 1, nz = 2 * mmax[2] + 1;
    long total = (long)nx * ny * nz;
    double U = 0, W[9] = {0}, Wr = 0;
    int nthr = 1;
#ifdef _OPENMP
    nthr = omp_get_max_threads();
#endif
    double *Ft = (double *)calloc((size_t)nthr * 3 * N, sizeof(double));
#pragma omp parallel
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *Fl = Ft + (size_t)tid * 3 * N;
        double u = 0, tw[9] = {0}, twr = 0;
#pragma omp for schedule(static)
        for (long id = 0; id < total; ++id) {
            int m[3] = {(int)(id % nx) - mmax[0], (int)((id / nx) % ny) - mmax[1],
                        (int)(id / ((long)nx * ny)) - mmax[2]};
            if (!m[0] && !m[1] && !m[2]) continue;
            double k[3];
            for (int a = 0; a < 3; ++a)
                k[a] = 2.0 * ORC_PI * (hi[a] * m[0] + hi[3 + a] * m[1] + hi[6 + a] * m[2]);
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double re = 0, im = 0;
            for (int j = 0; j < N; ++j) {
                double th = k[0] * r[3 * j] + k[1] * r[3 * j + 1] + k[2] * r[3 * j + 2];
                re += q[j] * cos(th);
                im += q[j] * sin(th);
            }
            double rho2 = re * re + im * im;
            double fhE = 0, fhF = 0, a5 = 0, a7 = 0;
            for (int l = 0; l < ME; ++l)
                fhE += pi15 * w[l] * s[l] * s[l] * s[l] * exp(-s[l] * s[l] * k2 / 4.0);
            for (int l = 0; l < M; ++l) {
                double e = exp(-st[l] * st[l] * k2 / 4.0);
                double s5 = st[l] * st[l] * st[l] * st[l] * st[l];
                fhF += 0.5 * pi15 * wt[l] * s5 * e;
                a5 += wt[l] * s5 * e;
                a7 += wt[l] * s5 * st[l] * st[l] * e;
            }
            u += ke * fhE * rho2 / (2.0 * V);
            twr += ke * pi15 / (4.0 * V) * a5 * rho2;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    tw[3 * a + b] += ke * pi15 / (4.0 * V) * ((a == b ? a5 : 0.0) - 0.5 * a7 * k[a] * k[b]) * rho2;
            for (int j = 0; j < N; ++j) {
                double th = k[0] * r[3 * j] + k[1] * r[3 * j + 1] + k[2] * r[3 * j + 2];
                /* Im(e^{-i th} rho) = im cos th - re sin th */
                double g = im * cos(th) - re * sin(th);
                double c = -ke * q[j] / V * fhF * g;
                Fl[3 * j] += c * k[0]; Fl[3 * j + 1] += c * k[1]; Fl[3 * j + 2] += c * k[2];
            }
        }
#pragma omp for ordered schedule(static, 1)
        for (int t = 0; t < orc_team_size(); ++t) {
#pragma omp ordered
            { U += u; Wr += twr; for (int a = 0; a < 9; ++a) W[a] += tw[a]; }
        }
    }
    for (int t = 0; t < nthr; ++t)
        for (long i = 0; i < 3L * N; ++i) F[i] += Ft[(size_t)t * 3 * N + i];
    free(Ft);
    UF[0] = U;
    for (int a = 0; a < 9; ++a) WF[a] = W[a];
    if (WFr) WFr[0] = Wr;   /* radial part (eq. PcoulFr): V P^F,r = WFr I */
}

/* eq. PFcoul for one Gaussian l: V P^F_l = (1/2) sum_n sum_{i,j} q_i q_j
 * w~_l e^{-|r_ij + h n|^2 / s~_l^2} (r_ij + h n) (x) (r_ij + h n), times ke,
 * images |n_a| <= nmax[a]. */
void orc_pf_realspace(int N, const double *r, const double *q, const double *h,
                      double wtl, double stl, const int *nmax, double ke, double *WF)
{
    double W[9] = {0};
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
                for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                    for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                        double d[3];
                        for (int a = 0; a < 3; ++a)
                            d[a] = r[3 * i + a] - r[3 * j + a] + h[3 * a] * n0 + h[3 * a + 1] * n1 + h[3 * a + 2] * n2;
                        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                        double g = 0.5 * ke * q[i] * q[j] * wtl * exp(-r2 / (stl * stl));
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) W[3 * a + b] += g * d[a] * d[b];
                    }
    for (int a = 0; a < 9; ++a) WF[a] = W[a];
}

/* ------------------------------------------------------------------------ */
/* normalizers S^r, S^nr (eqs. Sr, Snr) for an orthorhombic cell             */
/* ------------------------------------------------------------------------ */

/* 1D lattice sums along one axis for Gaussian l: with a = (pi s~ / L)^2,
 * S_n = sum_m m^n e^{-a m^2} (n = 0, 2, 4), |m| <= mmax = ceil(sqrt(46/a)) + 2. */
static int axis_mmax(double a) { return (int)ceil(sqrt(46.0 / a)) + 2; }

static void axis_sums(double stl, double L, double *S0, double *S2, double *S4)
{
    double c = ORC_PI * stl / L, a = c * c;
    int mm = axis_mmax(a);
    double s0 = 0, s2 = 0, s4 = 0;
    for (int m = -mm; m <= mm; ++m) {
        double m2 = (double)m * (double)m;
        double e = exp(-(a * m2));
        s0 += e; s2 += m2 * e; s4 += m2 * m2 * e;
    }
    *S0 = s0; *S2 = s2; *S4 = s4;
}

/* H^r_l = pi^1.5 w~ s~^5 sum_m |k|^2 e^{-s~^2|k|^2/4}; for an orthorhombic cell
 * e^{-s~^2|k|^2/4} factorises over the axes, so with T_n = (2 pi / L)^n S_n:
 *   H^r_l  = c_l  [T2x T0y T0z + T0x T2y T0z + T0x T0y T2z]
 *   H^nr_l = c'_l [sum_a T4a prod_{b!=a} T0b + 2 (T2x T2y T0z + T2x T0y T2z + T0x T2y T2z)]
 * with c_l = pi^1.5 w~ s~^5 and c'_l = pi^1.5 w~ s~^7 (k^4 = (sum k_a^2)^2).
 * T0/T2/T4 (3 x M each, axis fastest) are returned when non-null. */
void orc_normalizers(const double L[3], int M, const double *wt, const double *st,
                     double *Hr, double *Hnr, double *T0o, double *T2o, double *T4o)
{
    const double pi15 = pow(ORC_PI, 1.5);
    for (int l = 0; l < M; ++l) {
        double T0[3], T2[3], T4[3];
        for (int a = 0; a < 3; ++a) {
            double S0, S2, S4, g = 2.0 * ORC_PI / L[a];
            axis_sums(st[l], L[a], &S0, &S2, &S4);
            T0[a] = S0; T2[a] = g * g * S2; T4[a] = g * g * g * g * S4;
            if (T0o) { T0o[3 * l + a] = T0[a]; T2o[3 * l + a] = T2[a]; T4o[3 * l + a] = T4[a]; }
        }
        double s5 = pow(st[l], 5.0);
        double cr = pi15 * wt[l] * s5, cn = pi15 * wt[l] * s5 * st[l] * st[l];
        Hr[l] = cr * (T2[0] * T0[1] * T0[2] + T0[0] * T2[1] * T0[2] + T0[0] * T0[1] * T2[2]);
        Hnr[l] = cn * (T4[0] * T0[1] * T0[2] + T0[0] * T4[1] * T0[2] + T0[0] * T0[1] * T4[2]
                       + 2.0 * (T2[0] * T2[1] * T0[2] + T2[0] * T0[1] * T2[2] + T0[0] * T2[1] * T2[2]));
    }
}

/* eqs. Sr, Snr summed over m in Z^3 directly (|m_a| <= mmax[a]), general h. */
void orc_normalizers_3d(const double *h, int M, const double *wt, const double *st,
                        const int *mmax, double *Hr, double *Hnr)
{
    double hi[9];
    inv3(h, hi);
    const double pi15 = pow(ORC_PI, 1.5);
    for (int l = 0; l < M; ++l) {
        double sr = 0, snr = 0;
        for (int m0 = -mmax[0]; m0 <= mmax[0]; ++m0)
            for (int m1 = -mmax[1]; m1 <= mmax[1]; ++m1)
                for (int m2 = -mmax[2]; m2 <= mmax[2]; ++m2) {
                    double k[3];
                    for (int a = 0; a < 3; ++a)
                        k[a] = 2.0 * ORC_PI * (hi[a] * m0 + hi[3 + a] * m1 + hi[6 + a] * m2);
                    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    double e = exp(-st[l] * st[l] * k2 / 4.0);
                    sr += k2 * e;
                    snr += k2 * k2 * e;
                }
        double s5 = pow(st[l], 5.0);
        Hr[l] = pi15 * wt[l] * s5 * sr;
        Hnr[l] = pi15 * wt[l] * s5 * st[l] * st[l] * snr;
    }
}

/* Proposition 3.5: H^r_l = V w~ [6 A0 - 4 A2 / s~^2],
 * H^nr_l = V w~ [60 A0 - 80 A2 / s~^2 + 16 A4 / s~^4],
 * A_n = sum_{m in Z^3} |h m|^n e^{-|h m|^2 / s~^2}, summed directly over
 * |m_a| <= nmax[a] (general h). */
void orc_normalizers_poisson(const double *h, int M, const double *wt, const double *st,
                             const int *nmax, double *Hr, double *Hnr)
{
    const double V = fabs(det3(h));
    for (int l = 0; l < M; ++l) {
        double A0 = 0, A2 = 0, A4 = 0;
        for (int n0 = -nmax[0]; n0 <= nmax[0]; ++n0)
            for (int n1 = -nmax[1]; n1 <= nmax[1]; ++n1)
                for (int n2 = -nmax[2]; n2 <= nmax[2]; ++n2) {
                    double d[3];
                    for (int a = 0; a < 3; ++a) d[a] = h[3 * a] * n0 + h[3 * a + 1] * n1 + h[3 * a + 2] * n2;
                    double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                    double e = exp(-d2 / (st[l] * st[l]));
                    A0 += e; A2 += d2 * e; A4 += d2 * d2 * e;
                }
        double s2 = st[l] * st[l];
        Hr[l] = V * wt[l] * (6.0 * A0 - 4.0 * A2 / s2);
        Hnr[l] = V * wt[l] * (60.0 * A0 - 80.0 * A2 / s2 + 16.0 * A4 / (s2 * s2));
    }
}

/* ------------------------------------------------------------------------ */
/* mode sampling (App. D and sec. 3.2)                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    double L[3];
    int M;
    double wt[ORC_MAXM], st[ORC_MAXM];
    double cr[ORC_MAXM], cn[ORC_MAXM], st2q[ORC_MAXM];  /* pi^1.5 w~ s~^5, pi^1.5 w~ s~^7, s~^2/4 */
    double T0[3 * ORC_MAXM], T2[3 * ORC_MAXM], T4[3 * ORC_MAXM];
    double Hr[ORC_MAXM], Hnr[ORC_MAXM];
} modes_ctx;

static void modes_ctx_init(modes_ctx *c, const double L[3], int M, const double *wt, const double *st)
{
    const double pi15 = pow(ORC_PI, 1.5);
    memcpy(c->L, L, 3 * sizeof(double));
    c->M = M;
    for (int l = 0; l < M; ++l) {
        double s5 = st[l] * st[l] * st[l] * st[l] * st[l];
        c->wt[l] = wt[l]; c->st[l] = st[l];
        c->cr[l] = pi15 * wt[l] * s5;
        c->cn[l] = pi15 * wt[l] * s5 * st[l] * st[l];
        c->st2q[l] = st[l] * st[l] * 0.25;
    }
    orc_normalizers(L, M, wt, st, c->Hr, c->Hnr, c->T0, c->T2, c->T4);
}

/* unnormalised radial and non-radial targets (eqs. samplingP, samplingPnr):
 * pr = |k|^2 sum_l c_l e_l, pnr = |k|^4 sum_l c'_l e_l, e_l = exp(-(s~_l^2/4) |k|^2) */
static void targets(const modes_ctx *c, const int *m, double *pr, double *pnr)
{
    double kx = 2.0 * ORC_PI * m[0] / c->L[0];
    double ky = 2.0 * ORC_PI * m[1] / c->L[1];
    double kz = 2.0 * ORC_PI * m[2] / c->L[2];
    double k2 = kx * kx + ky * ky + kz * kz;
    double a = 0, b = 0;
    for (int l = 0; l < c->M; ++l) {
        double e = exp(-(c->st2q[l] * k2));
        a += c->cr[l] * e;
        b += c->cn[l] * e;
    }
    *pr = k2 * a;
    *pnr = (k2 * k2) * b;
}

/* eq. proposal for an orthorhombic cell: the Gaussian integral over the unit
 * cube around m factorises into 1D masses
 * q_a(m) = (1/2)[erf(pi s~0 (m+1/2)/L) - erf(pi s~0 (m-1/2)/L)],
 * written with erfc for |m| >= 1 (the same number without cancellation). */
static double q1d(int m, double L, double st0)
{
    double c = ORC_PI * st0 / L;
    int am = m < 0 ? -m : m;
    if (am == 0) return erf(c * 0.5);
    double lo = c * ((double)am - 0.5), hi = c * ((double)am + 0.5);
    return 0.5 * (erfc(lo) - erfc(hi));
}

static double qprop(const modes_ctx *c, const int *m)
{
    return q1d(m[0], c->L[0], c->st[0]) * q1d(m[1], c->L[1], c->st[0]) * q1d(m[2], c->L[2], c->st[0]);
}

/* one coordinate from the 1D law m^{2n} e^{-a m^2} on Z by inverse CDF,
 * visiting m = 0, 1, -1, 2, -2, ...; target = u * (the law's total). */
static int draw_axis(double u, double stl, double L, int n, double total)
{
    double c = ORC_PI * stl / L, a = c * c;
    int mm = axis_mmax(a);
    double target = u * total, cum = 0.0;
    int last = 0;
    for (int k = 0; k <= 2 * mm; ++k) {
        int m = (k == 0) ? 0 : ((k & 1) ? (k + 1) / 2 : -(k / 2));
        double m2 = (double)m * (double)m;
        double wgt = exp(-(a * m2));
        if (n >= 1) wgt *= m2;
        if (n >= 2) wgt *= m2;
        cum += wgt;
        last = m;
        if (cum > target) return m;
    }
    return last;
}

static double axis_total(const modes_ctx *c, int l, int a, int n)
{
    double g = 2.0 * ORC_PI / c->L[a];
    if (n == 0) return c->T0[3 * l + a];
    if (n == 1) return c->T2[3 * l + a] / (g * g);
    return c->T4[3 * l + a] / (g * g * g * g);
}

/* Exact draw from P^r: a mixture over (l, axis a) with weights
 * c_l T2_a prod_{b!=a} T0_b (the terms of H^r_l); inside a component the axis
 * a follows m^2 e^{-a m^2} and the others e^{-a m^2}.  Uses the four words of
 * one Philox block. */
static void exact_draw_r(const modes_ctx *c, const uint64_t wds[4], int *m)
{
    double tot = 0;
    for (int l = 0; l < c->M; ++l) tot += c->Hr[l];
    double target = orc_u01(wds[0]) * tot, cum = 0;
    int lsel = c->M - 1, asel = 2;
    for (int l = 0; l < c->M; ++l) {
        const double *T0 = c->T0 + 3 * l, *T2 = c->T2 + 3 * l;
        double comp[3] = {c->cr[l] * T2[0] * T0[1] * T0[2], c->cr[l] * T0[0] * T2[1] * T0[2],
                          c->cr[l] * T0[0] * T0[1] * T2[2]};
        int done = 0;
        for (int a = 0; a < 3; ++a) {
            cum += comp[a];
            if (cum > target) { lsel = l; asel = a; done = 1; break; }
        }
        if (done) break;
    }
    for (int a = 0; a < 3; ++a) {
        int n = (a == asel) ? 1 : 0;
        m[a] = draw_axis(orc_u01(wds[1 + a]), c->st[lsel], c->L[a], n, axis_total(c, lsel, a, n));
    }
}

/* Exact draw from P^nr: k^4 = sum_a k_a^4 + 2 sum_{a<b} k_a^2 k_b^2 gives six
 * components per l: (a, a) with weight c'_l T4_a prod T0 and (a, b) with
 * weight 2 c'_l T2_a T2_b T0_c. */
static void exact_draw_nr(const modes_ctx *c, const uint64_t wds[4], int *m)
{
    double tot = 0;
    for (int l = 0; l < c->M; ++l) tot += c->Hnr[l];
    double target = orc_u01(wds[0]) * tot, cum = 0;
    int lsel = c->M - 1, kind = 5;
    static const int pa[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
    for (int l = 0; l < c->M; ++l) {
        const double *T0 = c->T0 + 3 * l, *T2 = c->T2 + 3 * l, *T4 = c->T4 + 3 * l;
        double comp[6] = {c->cn[l] * T4[0] * T0[1] * T0[2], c->cn[l] * T0[0] * T4[1] * T0[2],
                          c->cn[l] * T0[0] * T0[1] * T4[2], 2.0 * c->cn[l] * T2[0] * T2[1] * T0[2],
                          2.0 * c->cn[l] * T2[0] * T0[1] * T2[2], 2.0 * c->cn[l] * T0[0] * T2[1] * T2[2]};
        int done = 0;
        for (int t = 0; t < 6; ++t) {
            cum += comp[t];
            if (cum > target) { lsel = l; kind = t; done = 1; break; }
        }
        if (done) break;
    }
    for (int a = 0; a < 3; ++a) {
        int n = pa[kind][a];
        m[a] = draw_axis(orc_u01(wds[1 + a]), c->st[lsel], c->L[a], n, axis_total(c, lsel, a, n));
    }
}

/* Philox purposes: counter = (step, purpose, index, 0), key = (seed, sysid). */
enum { PUR_START = 1, PUR_PROPOSAL = 2, PUR_ACCEPT = 3, PUR_NR_IID = 4, PUR_ATOM = 5, PUR_BOX = 6 };

/* Draw the P radial modes m^r and the P non-radial modes m^nr for one step.
 * kind 0 (the paper's construction):
 *   radial chain (App. D): x_0 is an exact draw from P^r (the paper leaves the
 *   start open); at t = 1..P propose m* = round(L_a u_a), u_a ~ N(0,
 *   1/(2 pi^2 s~0^2)), and accept with probability min{1, P^r(m*) q(x)/(P^r(x)
 *   q(m*))} (eq. acc_Gaussian), i.e. iff u_t w(x) < w(m*) with w = pr/q
 *   (pr(0) = 0: m* = 0 is never accepted); m^r_t = x_t.
 *   recalibration chain (sec. 3.2): y_0 = x_1; at t = 1..P propose x_t and
 *   accept iff u'_t g(y) < g(x_t), g = pnr/pr (the ratio of eq. Acc with the
 *   state-independent proposal P^r); m^nr_t = y_t.
 * kind 1: m^r and m^nr are independent exact draws from P^r and P^nr.
 * kind 2: m^r are independent exact draws from P^r and the recalibration
 *   chain above runs on them, started from an exact P^nr draw: with i.i.d.
 *   P^r proposals every y_t is exactly P^nr-distributed (kind 0's radial
 *   states are serially correlated, which biases its y_t; a property of the
 *   construction, measured in the tests).
 * stats[0..1] = accepted moves of the two chains. */
void orc_sample_modes(const double L[3], int M, const double *wt, const double *st,
                      int P, uint64_t seed, uint64_t sysid, uint64_t step, int kind,
                      int *mr, int *mnr, double *stats)
{
    modes_ctx *c = (modes_ctx *)malloc(sizeof(modes_ctx));
    modes_ctx_init(c, L, M, wt, st);
    uint64_t wds[4];
    stats[0] = stats[1] = 0;
    if (kind == 1) {
        for (int t = 0; t < P; ++t) {
            draw4(seed, sysid, step, PUR_START, (uint64_t)t, wds);
            exact_draw_r(c, wds, mr + 3 * t);
            draw4(seed, sysid, step, PUR_NR_IID, (uint64_t)t, wds);
            exact_draw_nr(c, wds, mnr + 3 * t);
        }
        free(c);
        return;
    }
    const double sig_u = 1.0 / (sqrt(2.0) * ORC_PI * st[0]);
    int x[3];
    double pr, pnr;
    if (kind == 2) {
        /* exact i.i.d. radial draws in place of the App. D chain */
        for (int t = 0; t < P; ++t) {
            draw4(seed, sysid, step, PUR_START, (uint64_t)t, wds);
            exact_draw_r(c, wds, mr + 3 * t);
        }
        goto recalibrate;
    }
    draw4(seed, sysid, step, PUR_START, 0, wds);
    exact_draw_r(c, wds, x);
    targets(c, x, &pr, &pnr);
    double wcur = pr / qprop(c, x);
    for (int t = 1; t <= P; ++t) {
        double z[3], zz;
        draw4(seed, sysid, step, PUR_PROPOSAL, (uint64_t)(t - 1), wds);
        box_muller(wds[0], wds[1], &z[0], &z[1]);
        box_muller(wds[2], wds[3], &z[2], &zz);
        int ms[3];
        for (int a = 0; a < 3; ++a) ms[a] = (int)floor(L[a] * (z[a] * sig_u) + 0.5);
        double ws = 0.0;
        if (ms[0] || ms[1] || ms[2]) {
            targets(c, ms, &pr, &pnr);
            ws = pr / qprop(c, ms);
        }
        draw4(seed, sysid, step, PUR_ACCEPT, (uint64_t)(t - 1), wds);
        if (orc_u01(wds[0]) * wcur < ws) {
            x[0] = ms[0]; x[1] = ms[1]; x[2] = ms[2];
            wcur = ws;
            stats[0] += 1;
        }
        mr[3 * (t - 1)] = x[0]; mr[3 * (t - 1) + 1] = x[1]; mr[3 * (t - 1) + 2] = x[2];
    }
recalibrate:;
    int y[3] = {mr[0], mr[1], mr[2]};
    if (kind == 2) {
        /* start the recalibration chain from an exact P^nr draw */
        draw4(seed, sysid, step, PUR_NR_IID, 0, wds);
        exact_draw_nr(c, wds, y);
    }
    targets(c, y, &pr, &pnr);
    double gcur = pnr / pr;
    for (int t = 1; t <= P; ++t) {
        const int *xt = mr + 3 * (t - 1);
        targets(c, xt, &pr, &pnr);
        double gt = pnr / pr;
        draw4(seed, sysid, step, PUR_ACCEPT, (uint64_t)(t - 1), wds);
        if (orc_u01(wds[1]) * gcur < gt) {
            y[0] = xt[0]; y[1] = xt[1]; y[2] = xt[2];
            gcur = gt;
            stats[1] += 1;
        }
        mnr[3 * (t - 1)] = y[0]; mnr[3 * (t - 1) + 1] = y[1]; mnr[3 * (t - 1) + 2] = y[2];
    }
    free(c);
}

/* exported pieces of the sampler, for tests */
void orc_targets(const double L[3], int M, const double *wt, const double *st,
                 const int *m, double *out /* pr, pnr, q */)
{
    modes_ctx *c = (modes_ctx *)malloc(sizeof(modes_ctx));
    modes_ctx_init(c, L, M, wt, st);
    targets(c, m, &out[0], &out[1]);
    out[2] = qprop(c, m);
    free(c);
}

static int cmp_mode(const void *a, const void *b)
{
    const int *x = (const int *)a, *y = (const int *)b;
    for (int k = 0; k < 3; ++k)
        if (x[k] != y[k]) return x[k] < y[k] ? -1 : 1;
    return 0;
}

/* sec. 3.2: the distinct modes D of {m^r} u {m^nr} in lexicographic order
 * (m_x, m_y, m_z), with multiplicities c_r[d], c_nr[d].  Returns |D|. */
int orc_distinct(int P, const int *mr, int Pn, const int *mnr, int *D, int *cr, int *cnr)
{
    int n = P + Pn;
    int *all = (int *)malloc(sizeof(int) * 3 * (size_t)n);
    memcpy(all, mr, sizeof(int) * 3 * (size_t)P);
    memcpy(all + 3 * P, mnr, sizeof(int) * 3 * (size_t)Pn);
    qsort(all, (size_t)n, 3 * sizeof(int), cmp_mode);
    int nd = 0;
    for (int i = 0; i < n; ++i) {
        if (nd == 0 || cmp_mode(all + 3 * i, D + 3 * (nd - 1)) != 0) {
            memcpy(D + 3 * nd, all + 3 * i, 3 * sizeof(int));
            nd++;
        }
    }
    for (int d = 0; d < nd; ++d) cr[d] = cnr[d] = 0;
    for (int i = 0; i < P; ++i) {
        int *hit = (int *)bsearch(mr + 3 * i, D, (size_t)nd, 3 * sizeof(int), cmp_mode);
        cr[(hit - D) / 3]++;
    }
    for (int i = 0; i < Pn; ++i) {
        int *hit = (int *)bsearch(mnr + 3 * i, D, (size_t)nd, 3 * sizeof(int), cmp_mode);
        cnr[(hit - D) / 3]++;
    }
    free(all);
    return nd;
}

/* eq. rho_k with k = 2 pi m / L (orthorhombic): rho = sum_j q_j e^{i k.r_j};
 * rho[2d] = Re, rho[2d+1] = Im. */
void orc_rho(int N, const double *r, const double *q, const double L[3], int nD,
             const int *D, double *rho)
{
#pragma omp parallel for schedule(static)
    for (int d = 0; d < nD; ++d) {
        double k[3];
        for (int a = 0; a < 3; ++a) k[a] = 2.0 * ORC_PI * D[3 * d + a] / L[a];
        double re = 0, im = 0;
        for (int j = 0; j < N; ++j) {
            double th = k[0] * r[3 * j] + k[1] * r[3 * j + 1] + k[2] * r[3 * j + 2];
            re += q[j] * cos(th);
            im += q[j] * sin(th);
        }
        rho[2 * d] = re;
        rho[2 * d + 1] = im;
    }
}

/* Random batch estimators (sec. 3.2, App. B) over the distinct modes with
 * multiplicities (P radial and P non-radial samples):
 *   U^F*     = ke S^r /(4 V P) sum_d c_r |rho_d|^2 / k_d^2    (App. A energy with
 *              the force proposal P = P^r and S = S^r / 2 of App. B)
 *   V P^F,r* = ke S^r /(4 V P) sum_d c_r |rho_d|^2 / k_d^2 I     (eq. P_approx_r)
 *   V P^F,nr*= -ke S^nr/(8 V P) sum_d c_nr |rho_d|^2 k (x) k / k^4 (eq. P_approx_nr)
 *   F_i     += -ke (S^r/2)/P (q_i/V) sum_d c_r k_d Im(e^{-ik.r_i} rho_d)/k_d^2
 *                                                            (eq. f_approx)
 * rho is computed here (orc_rho).  out[0] = U^F*; Wr, Wnr = the virials
 * V P^F,r* and V P^F,nr* (kcal/mol). */
void orc_rb_longrange(int N, const double *r, const double *q, const double L[3],
                      int P, int nD, const int *D, const int *cr, const int *cnr,
                      double Sr, double Snr, double ke, double *F, double *out,
                      double *Wr, double *Wnr, double *rho)
{
    const double V = L[0] * L[1] * L[2];
    orc_rho(N, r, q, L, nD, D, rho);
    double Ar = 0, B[9] = {0};
    for (int d = 0; d < nD; ++d) {
        double k[3];
        for (int a = 0; a < 3; ++a) k[a] = 2.0 * ORC_PI * D[3 * d + a] / L[a];
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double r2 = rho[2 * d] * rho[2 * d] + rho[2 * d + 1] * rho[2 * d + 1];
        Ar += cr[d] * r2 / k2;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) B[3 * a + b] += cnr[d] * r2 * k[a] * k[b] / (k2 * k2);
    }
    out[0] = ke * Sr / (4.0 * V * P) * Ar;
    for (int a = 0; a < 9; ++a) {
        Wr[a] = (a % 4 == 0) ? ke * Sr / (4.0 * V * P) * Ar : 0.0;
        Wnr[a] = -ke * Snr / (8.0 * V * P) * B[a];
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double f[3] = {0, 0, 0};
        for (int d = 0; d < nD; ++d) {
            if (!cr[d]) continue;
            double k[3];
            for (int a = 0; a < 3; ++a) k[a] = 2.0 * ORC_PI * D[3 * d + a] / L[a];
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double th = k[0] * r[3 * i] + k[1] * r[3 * i + 1] + k[2] * r[3 * i + 2];
            double g = rho[2 * d + 1] * cos(th) - rho[2 * d] * sin(th);
            for (int a = 0; a < 3; ++a) f[a] += cr[d] * k[a] * g / k2;
        }
        double c = -ke * (0.5 * Sr) / P * q[i] / V;
        for (int a = 0; a < 3; ++a) F[3 * i + a] += c * f[a];
    }
}

/* Shared-proposal estimator of the non-radial virial (sec. 3.2, the
 * alternative the measure recalibration replaces): the P radial samples of
 * P^r (eq. samplingP) are reused for eq. PcoulFnr with importance weight
 * f_nr(k) / P^r(k) = S^r k^2 R(k), where f_nr is the unnormalised P^nr of
 * eq. samplingPnr and R(k) = sum_l w~_l s~_l^7 e^{-s~_l^2 k^2/4} /
 * sum_l w~_l s~_l^5 e^{-s~_l^2 k^2/4}:
 *   V P^F,nr,sh = -ke S^r /(8 V P) sum_d c_r R(k_d) |rho_d|^2 k (x) k / k^2.
 * rho as returned by orc_rb_longrange (or orc_rho).  W: 9 values, kcal/mol. */
void orc_nr_shared(const double L[3], int P, int nD, const int *D, const int *cr, const double *rho,
                   int M, const double *wt, const double *st, double Sr, double ke, double *W)
{
    const double V = L[0] * L[1] * L[2];
    double B[9] = {0};
    for (int d = 0; d < nD; ++d) {
        if (!cr[d]) continue;
        double k[3];
        for (int a = 0; a < 3; ++a) k[a] = 2.0 * ORC_PI * D[3 * d + a] / L[a];
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double num = 0, den = 0;
        for (int l = 0; l < M; ++l) {
            double e = exp(-st[l] * st[l] * k2 / 4.0);
            double s5 = pow(st[l], 5);
            den += wt[l] * s5 * e;
            num += wt[l] * s5 * st[l] * st[l] * e;
        }
        double r2 = rho[2 * d] * rho[2 * d] + rho[2 * d + 1] * rho[2 * d + 1];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) B[3 * a + b] += cr[d] * (num / den) * r2 * k[a] * k[b] / k2;
    }
    for (int a = 0; a < 9; ++a) W[a] = -ke * Sr / (8.0 * V * P) * B[a];
}

/* App. A: U_self = ln b /(sqrt(2 pi) sigma) (omega + (1 - b^{-(M-1)})/(b - 1)) sum q^2, times ke. */
double orc_self_energy(double b, double sigma, double omega, int ME, int N, const double *q, double ke)
{
    double sq = 0;
    for (int i = 0; i < N; ++i) sq += q[i] * q[i];
    return ke * log(b) / (sqrt(2.0 * ORC_PI) * sigma) * (omega + (1.0 - pow(b, -(ME - 1.0))) / (b - 1.0)) * sq;
}

/* Intramolecular (excluded) pairs: the Fourier part holds their long-range
 * interaction q_i q_j F(r); remove it: U -= ke q_i q_j F_E(r),
 * f_i = -ke q_i q_j F~(r) r_ij (F'(r)/r = -F~(r) for w = w~ s~^2/2),
 * virial += f_i (x) r_ij. */
void orc_exclusions(int ne, const int *pairs, const double *r, const double *q, const double *h,
                    int M, const double *wt, const double *st, int ME, const double *w, const double *s,
                    double ke, double *F, double *U, double *W)
{
    double hi[9], u = 0, t[9] = {0};
    inv3(h, hi);
    for (int e = 0; e < ne; ++e) {
        int i = pairs[2 * e], j = pairs[2 * e + 1];
        double d[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
        min_image(h, hi, d);
        double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double fe = 0, ft = 0;
        for (int l = 0; l < ME; ++l) fe += w[l] * exp(-r2 / (s[l] * s[l]));
        for (int l = 0; l < M; ++l) ft += wt[l] * exp(-r2 / (st[l] * st[l]));
        double qq = ke * q[i] * q[j];
        u -= qq * fe;
        for (int a = 0; a < 3; ++a) {
            double f = -qq * ft * d[a];
            F[3 * i + a] += f;
            F[3 * j + a] -= f;
            for (int b = 0; b < 3; ++b) t[3 * a + b] += f * d[b];
        }
    }
    U[0] = u;
    for (int a = 0; a < 9; ++a) W[a] = t[a];
}

/* Harmonic bonds U = k (r - r0)^2 and angles U = k (theta - theta0)^2
 * (minimum image); en[0] = bonds, en[1] = angles; W = virial. */
void orc_bonded(int nb, const int *bonds, const double *bk, const double *br0,
                int na, const int *angles, const double *ak, const double *at0,
                const double *r, const double *h, double *F, double *en, double *W)
{
    double hi[9], ub = 0, ua = 0, t[9] = {0};
    inv3(h, hi);
    for (int e = 0; e < nb; ++e) {
        int i = bonds[2 * e], j = bonds[2 * e + 1];
        double d[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
        min_image(h, hi, d);
        double rr = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double dr = rr - br0[e];
        ub += bk[e] * dr * dr;
        double c = -2.0 * bk[e] * dr / rr;
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += c * d[a];
            F[3 * j + a] -= c * d[a];
            for (int b = 0; b < 3; ++b) t[3 * a + b] += c * d[a] * d[b];
        }
    }
    for (int e = 0; e < na; ++e) {
        int i = angles[3 * e], j = angles[3 * e + 1], k = angles[3 * e + 2];
        double d1[3] = {r[3 * i] - r[3 * j], r[3 * i + 1] - r[3 * j + 1], r[3 * i + 2] - r[3 * j + 2]};
        double d2[3] = {r[3 * k] - r[3 * j], r[3 * k + 1] - r[3 * j + 1], r[3 * k + 2] - r[3 * j + 2]};
        min_image(h, hi, d1);
        min_image(h, hi, d2);
        double r1 = sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        double r2 = sqrt(d2[0] * d2[0] + d2[1] * d2[1] + d2[2] * d2[2]);
        double cs = (d1[0] * d2[0] + d1[1] * d2[1] + d1[2] * d2[2]) / (r1 * r2);
        if (cs > 1.0) cs = 1.0;
        if (cs < -1.0) cs = -1.0;
        double th = acos(cs), sn = sqrt(1.0 - cs * cs);
        if (sn < 1e-12) sn = 1e-12;
        double dth = th - at0[e];
        ua += ak[e] * dth * dth;
        double g = 2.0 * ak[e] * dth / sn;   /* -dU/dtheta * dtheta/dcos = (dU/dtheta)/sin */
        double fi[3], fk[3];
        for (int a = 0; a < 3; ++a) {
            fi[a] = g * (d2[a] / (r1 * r2) - cs * d1[a] / (r1 * r1));
            fk[a] = g * (d1[a] / (r1 * r2) - cs * d2[a] / (r2 * r2));
        }
        for (int a = 0; a < 3; ++a) {
            F[3 * i + a] += fi[a];
            F[3 * k + a] += fk[a];
            F[3 * j + a] -= fi[a] + fk[a];
            for (int b = 0; b < 3; ++b) t[3 * a + b] += fi[a] * d1[b] + fk[a] * d2[b];
        }
    }
    en[0] = ub; en[1] = ua;
    for (int a = 0; a < 9; ++a) W[a] = t[a];
}

/* ------------------------------------------------------------------------ */
/* one full force evaluation and the NPT integrator                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    double rc, b, sigma, omega, ke;
    int M, ME, P, kind;
    uint64_t seed, sysid;
    int short_cells;              /* 1: short range over cell lists (same results; timed baseline) */
} orc_params;

typedef struct {
    int N;
    const double *q, *mass;
    const int *type, *mol;
    int ntypes;
    const double *lj_eps, *lj_sig;
    int nb; const int *bonds; const double *bk, *br0;
    int na; const int *angles; const double *ak, *at0;
    int ne; const int *excl;
} orc_system;

/* Algorithm 1, steps 2-7, for one configuration: forces F (overwritten),
 * en[0..8] = {U^N_coul, U^F*, U_self, U_excl, U_LJ, U_bond, U_angle, U_coul total, |D|},
 * W[9] = total virial (kcal/mol; V P without the kinetic part), Wparts[5*9] =
 * {short-range Coulomb, V P^F,r*, V P^F,nr*, LJ, bonded + exclusions}.
 * modes_out (optional, >= 6P ints) receives m^r then m^nr. */
void orc_force_eval(const orc_params *pp, const orc_system *sy, const double *r,
                    const double L[3], uint64_t step, double *F, double *en, double *W,
                    double *Wparts, int *modes_out)
{
    int N = sy->N, M = pp->M, ME = pp->ME, P = pp->P;
    int MM = M > ME ? M : ME;
    double *w = (double *)malloc(sizeof(double) * 4 * MM);
    double *s = w + MM, *wt = w + 2 * MM, *st = w + 3 * MM;
    orc_sog_terms(pp->b, pp->sigma, pp->omega, MM, w, s, wt, st);
    double h[9];
    diag_box(L, h);
    memset(F, 0, sizeof(double) * 3 * N);
    double esr[2], Wc[9], Wl[9];
    if (!pp->short_cells ||
        orc_short_range_cells(N, r, sy->q, sy->type, sy->mol, h, pp->rc, M, wt, st, ME, w, s,
                              sy->ntypes, sy->lj_eps, sy->lj_sig, pp->ke, F, esr, Wc, Wl) != 0)
        orc_short_range(N, r, sy->q, sy->type, sy->mol, h, pp->rc, M, wt, st, ME, w, s,
                        sy->ntypes, sy->lj_eps, sy->lj_sig, pp->ke, F, esr, Wc, Wl);
    int *mr = (int *)malloc(sizeof(int) * 6 * P);
    int *mnr = mr + 3 * P;
    double stats[2];
    orc_sample_modes(L, M, wt, st, P, pp->seed, pp->sysid, step, pp->kind, mr, mnr, stats);
    if (modes_out) memcpy(modes_out, mr, sizeof(int) * 6 * P);
    int *D = (int *)malloc(sizeof(int) * 3 * 2 * P);
    int *cr = (int *)malloc(sizeof(int) * 2 * P), *cnr = (int *)malloc(sizeof(int) * 2 * P);
    int nD = orc_distinct(P, mr, P, mnr, D, cr, cnr);
    double Hr[ORC_MAXM], Hnr[ORC_MAXM], Sr = 0, Snr = 0;
    orc_normalizers(L, M, wt, st, Hr, Hnr, NULL, NULL, NULL);
    for (int l = 0; l < M; ++l) { Sr += Hr[l]; Snr += Hnr[l]; }
    double *rho = (double *)malloc(sizeof(double) * 2 * nD);
    double uf, Wr[9], Wnr[9];
    orc_rb_longrange(N, r, sy->q, L, P, nD, D, cr, cnr, Sr, Snr, pp->ke, F, &uf, Wr, Wnr, rho);
    double ux, Wx[9], eb[2], Wb[9];
    orc_exclusions(sy->ne, sy->excl, r, sy->q, h, M, wt, st, ME, w, s, pp->ke, F, &ux, Wx);
    orc_bonded(sy->nb, sy->bonds, sy->bk, sy->br0, sy->na, sy->angles, sy->ak, sy->at0, r, h, F, eb, Wb);
    double us = orc_self_energy(pp->b, pp->sigma, pp->omega, ME, N, sy->q, pp->ke);
    en[0] = esr[0]; en[1] = uf; en[2] = us; en[3] = ux; en[4] = esr[1]; en[5] = eb[0]; en[6] = eb[1];
    en[7] = esr[0] + uf - us + ux;
    en[8] = nD;
    for (int a = 0; a < 9; ++a) {
        W[a] = Wc[a] + Wr[a] + Wnr[a] + Wl[a] + Wx[a] + Wb[a];
        if (Wparts) {
            Wparts[a] = Wc[a]; Wparts[9 + a] = Wr[a]; Wparts[18 + a] = Wnr[a];
            Wparts[27 + a] = Wl[a]; Wparts[36 + a] = Wx[a] + Wb[a];
        }
    }
    free(rho); free(D); free(cr); free(cnr); free(mr); free(w);
}

typedef struct {
    double dt, T, Pext_atm, gamma, gamma_box;
    int coupling;                 /* 0 iso (one group), 1 semi-iso (xy, z) */
    double Mbox[3];               /* box mass per group (g/mol) */
    double kB, ftm2v, nktv2p;     /* kcal/(mol K); (kcal/mol/A)/(g/mol) -> A/fs^2; atm per kcal/mol/A^3 */
} orc_integ;

static int ngroups(int coupling) { return coupling == 0 ? 1 : (coupling == 1 ? 2 : 3); }
static int axis_group(int coupling, int a)
{
    if (coupling == 0) return 0;
    if (coupling == 1) return a == 2 ? 1 : 0;
    return a;
}

/* Generalised box force of eq. Langevin_NPT for a diagonal h restricted to
 * the coupled axes: G_g = sum_{a in g} (K_aa + W_aa - P_ext V - kB T) / L_a. */
static void box_force(const orc_integ *ig, const double L[3], const double *K, const double *W, double *G)
{
    double V = L[0] * L[1] * L[2];
    double pext = ig->Pext_atm / ig->nktv2p;
    G[0] = G[1] = G[2] = 0;
    for (int a = 0; a < 3; ++a)
        G[axis_group(ig->coupling, a)] += (K[4 * a] + W[4 * a] - pext * V - ig->kB * ig->T) / L[a];
}

static void kinetic(int N, const double *p, const double *mass, double mvv2e, double *K)
{
    for (int a = 0; a < 9; ++a) K[a] = 0;
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) K[3 * a + b] += p[3 * i + a] * p[3 * i + b] / mass[i];
    for (int a = 0; a < 9; ++a) K[a] *= mvv2e;
}

/* A: exact flow of dr/dt = p/m + (Ldot/L) r, dp/dt = -(Ldot/L) p with the box
 * velocity held: L' = L + v tau, r' = (L'/L) r + (p/m) tau, p' = (L/L') p. */
static void drift(const orc_integ *ig, int N, double *r, double *p, const double *mass,
                  double L[3], const double *ph, double tau)
{
    double Ln[3], sc[3];
    for (int a = 0; a < 3; ++a) {
        int g = axis_group(ig->coupling, a);
        double v = ig->Mbox[g] > 0.0 ? ph[g] / ig->Mbox[g] : 0.0;   /* Mbox <= 0: fixed box */
        Ln[a] = L[a] + v * tau;
        sc[a] = Ln[a] / L[a];
    }
    for (int i = 0; i < N; ++i)
        for (int a = 0; a < 3; ++a) {
            r[3 * i + a] = sc[a] * r[3 * i + a] + p[3 * i + a] / mass[i] * tau;
            p[3 * i + a] = p[3 * i + a] / sc[a];
        }
    for (int a = 0; a < 3; ++a) L[a] = Ln[a];
}

/* Algorithm 1 step 8: BAOAB splitting of eq. Langevin_NPT (the paper defers
 * its integrator to another work; this splitting is our reading):
 *   B  p^h += dt/2 G(K, W) ftm2v;  p += dt/2 F ftm2v
 *   A  dt/2 drift (box and atoms)
 *   O  p  <- c p + sqrt((1-c^2) m kB T ftm2v) xi,   c = exp(-gamma dt)
 *      p^h<- c_h p^h + sqrt((1-c_h^2) M kB T ftm2v) xi_h
 *   A  dt/2 drift;  wrap r into [0, L)
 *   force evaluation with step counter n
 *   B  p += dt/2 F ftm2v;  K = sum p p / m;  p^h += dt/2 G(K, W) ftm2v
 * State: r, p (g/mol A/fs), L, ph[3], F, W (from the last evaluation at
 * counter step0); runs steps step0+1 .. step0+nsteps.  A group with box
 * mass <= 0 keeps its box lengths fixed.  en_out (9) and W/K
 * (9 each) hold the last evaluation. */
void orc_npt_run(const orc_params *pp, const orc_system *sy, const orc_integ *ig,
                 double *r, double *p, double *L, double *ph, double *F, double *W,
                 uint64_t step0, int nsteps, double *en_out, double *K_out)
{
    int N = sy->N;
    double mvv2e = 1.0 / ig->ftm2v, K[9], G[3];
    double c = exp(-ig->gamma * ig->dt), ch = exp(-ig->gamma_box * ig->dt);
    int ng = ngroups(ig->coupling);
    kinetic(N, p, sy->mass, mvv2e, K);
    for (int n = 1; n <= nsteps; ++n) {
        uint64_t step = step0 + (uint64_t)n;
        box_force(ig, L, K, W, G);
        for (int g = 0; g < ng; ++g)
            if (ig->Mbox[g] > 0.0) ph[g] += 0.5 * ig->dt * G[g] * ig->ftm2v;
        for (int i = 0; i < 3 * N; ++i) p[i] += 0.5 * ig->dt * F[i] * ig->ftm2v;
        drift(ig, N, r, p, sy->mass, L, ph, 0.5 * ig->dt);
        uint64_t wds[4];
        for (int i = 0; i < N; ++i) {
            double z[4];
            draw4(pp->seed, pp->sysid, step, PUR_ATOM, (uint64_t)i, wds);
            box_muller(wds[0], wds[1], &z[0], &z[1]);
            box_muller(wds[2], wds[3], &z[2], &z[3]);
            double sdv = sqrt((1.0 - c * c) * sy->mass[i] * ig->kB * ig->T * ig->ftm2v);
            for (int a = 0; a < 3; ++a) p[3 * i + a] = c * p[3 * i + a] + sdv * z[a];
        }
        draw4(pp->seed, pp->sysid, step, PUR_BOX, 0, wds);
        {
            double z[4];
            box_muller(wds[0], wds[1], &z[0], &z[1]);
            box_muller(wds[2], wds[3], &z[2], &z[3]);
            for (int g = 0; g < ng; ++g) {
                if (ig->Mbox[g] <= 0.0) continue;
                double sdv = sqrt((1.0 - ch * ch) * ig->Mbox[g] * ig->kB * ig->T * ig->ftm2v);
                ph[g] = ch * ph[g] + sdv * z[g];
            }
        }
        drift(ig, N, r, p, sy->mass, L, ph, 0.5 * ig->dt);
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) {
                double x = r[3 * i + a];
                x -= L[a] * floor(x / L[a]);
                if (x >= L[a]) x -= L[a];
                r[3 * i + a] = x;
            }
        orc_force_eval(pp, sy, r, L, step, F, en_out, W, NULL, NULL);
        for (int i = 0; i < 3 * N; ++i) p[i] += 0.5 * ig->dt * F[i] * ig->ftm2v;
        kinetic(N, p, sy->mass, mvv2e, K);
        box_force(ig, L, K, W, G);
        for (int g = 0; g < ng; ++g)
            if (ig->Mbox[g] > 0.0) ph[g] += 0.5 * ig->dt * G[g] * ig->ftm2v;
    }
    for (int a = 0; a < 9; ++a) K_out[a] = K[a];
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* a general (triclinic) cell h                                              */
/* ------------------------------------------------------------------------ */
/*
 * h is upper triangular (the cell vectors a = (h00, 0, 0), b = (h01, h11, 0),
 * c = (h02, h12, h22) are its columns, the LAMMPS convention; any cell can be
 * rotated into this form).  The reciprocal vectors of eq. Sr are
 * k = 2 pi h^{-T} m, i.e. h^T k = 2 pi m, solved by forward substitution.
 *
 * Sampling (App. D with a general h):
 *   - proposal m* = round(h^T u), u_a ~ N(0, sigma_u^2), sigma_u^2 = 1/(2 pi^2 s~0^2);
 *   - its mass q(m*) (eq. proposal) is the probability that h^T u lies in the
 *     unit cube around m*.  With h^T lower triangular, (h^T u)_0 depends on
 *     u_0 only, (h^T u)_1 on u_0, u_1: the cube condition is an interval for
 *     u_0, an interval for u_1 given u_0 and one for u_2 given (u_0, u_1).  The
 *     u_2 integral is an erf difference; the (u_0, u_1) integral is taken by
 *     Gauss-Legendre quadrature with nq nodes per axis (nq = 20: converged to
 *     about 1e-15 relative for the boxes used, pinned in the tests);
 *   - the radial chain starts from an exact draw of P^r: component (l, a)
 *     with weight c_l sum_m k_a^2 e_l(m) (c_l = pi^1.5 w~ s~^5, e_l = e^{-s~_l^2
 *     k^2/4}; the weights over a add up to H^r_l), then m_0 from its marginal,
 *     m_1 given m_0 and m_2 given (m_0, m_1), each by inverse CDF over
 *     m = 0, 1, -1, 2, -2, ...  The sums run over |m_a| <= mm_a, the box that
 *     holds the ellipsoid |k| <= 2 sqrt(46)/s~0 (terms beyond it are below
 *     e^-46 of the largest).  For a diagonal h each step reduces to the
 *     orthorhombic draw (orc_sample_modes), which a test checks;
 *   - acceptance tests and the recalibration chain are those of
 *     orc_sample_modes with the general k.
 * Only the paper's construction (kind 0) is provided for a general h.
 */

static void kvec_h(const double *h, const int *m, double *k)
{
    k[0] = (2.0 * ORC_PI * (double)m[0]) / h[0];
    k[1] = (2.0 * ORC_PI * (double)m[1] - h[1] * k[0]) / h[4];
    k[2] = (2.0 * ORC_PI * (double)m[2] - h[2] * k[0] - h[5] * k[1]) / h[8];
}

/* Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n from
 * the Chebyshev-like first guess cos(pi (i + 3/4) / (n + 1/2)). */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = cos(ORC_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

/* P(lo <= u <= hi) for u ~ N(0, sig^2), without cancellation in the tails */
static double normal_interval(double lo, double hi, double sig)
{
    double x = lo / (sqrt(2.0) * sig), y = hi / (sqrt(2.0) * sig);
    if (x >= 0.0) return 0.5 * (erfc(x) - erfc(y));
    if (y <= 0.0) return 0.5 * (erfc(-y) - erfc(-x));
    return 0.5 * (erf(y) - erf(x));
}

/* eq. proposal for a general (upper-triangular) h: see the section comment. */
double orc_tri_q(const double *h, double st0, const int *m, int nq)
{
    double x[64], wq[64];
    if (nq < 1) nq = 1;
    if (nq > 64) nq = 64;
    gauss_legendre(nq, x, wq);
    const double sig = 1.0 / (sqrt(2.0) * ORC_PI * st0);
    const double nrm = 1.0 / (sqrt(2.0 * ORC_PI) * sig);
    const double A0 = ((double)m[0] - 0.5) / h[0], B0 = ((double)m[0] + 0.5) / h[0];
    double tot = 0.0;
    for (int i = 0; i < nq; ++i) {
        double u0 = 0.5 * (A0 + B0) + 0.5 * (B0 - A0) * x[i];
        double A1 = ((double)m[1] - 0.5 - h[1] * u0) / h[4], B1 = ((double)m[1] + 0.5 - h[1] * u0) / h[4];
        double inner = 0.0;
        for (int j = 0; j < nq; ++j) {
            double u1 = 0.5 * (A1 + B1) + 0.5 * (B1 - A1) * x[j];
            double c = h[2] * u0 + h[5] * u1;
            double pz = normal_interval(((double)m[2] - 0.5 - c) / h[8], ((double)m[2] + 0.5 - c) / h[8], sig);
            inner += wq[j] * nrm * exp(-u1 * u1 / (2.0 * sig * sig)) * pz;
        }
        tot += wq[i] * nrm * exp(-u0 * u0 / (2.0 * sig * sig)) * 0.5 * (B1 - A1) * inner;
    }
    return tot * 0.5 * (B0 - A0);
}

typedef struct {
    double h[9];
    int M, mm[3], nx, ny, nz;
    double wt[ORC_MAXM], st[ORC_MAXM], cr[ORC_MAXM], cn[ORC_MAXM], st2q[ORC_MAXM];
    double Hr[ORC_MAXM], Hnr[ORC_MAXM];
    double S[ORC_MAXM][3];     /* sum_m k_a^2 e_l(m) */
    double *Gx;                /* [M][3][nx]: sum over (m_1, m_2) of k_a^2 e_l */
    double *Gy;                /* [M][3][nx][ny]: sum over m_2 of k_a^2 e_l */
} tri_ctx;

static int walk_index(int k) { return (k == 0) ? 0 : ((k & 1) ? (k + 1) / 2 : -(k / 2)); }

/* Set up the sums of a cell h (upper triangular) and SOG split (w~, s~). */
tri_ctx *orc_tri_create(const double *h, int M, const double *wt, const double *st)
{
    if (M < 1 || M > ORC_MAXM || h[3] != 0.0 || h[6] != 0.0 || h[7] != 0.0) return NULL;
    tri_ctx *c = (tri_ctx *)calloc(1, sizeof(tri_ctx));
    memcpy(c->h, h, 9 * sizeof(double));
    c->M = M;
    const double pi15 = pow(ORC_PI, 1.5);
    for (int l = 0; l < M; ++l) {
        double s5 = st[l] * st[l] * st[l] * st[l] * st[l];
        c->wt[l] = wt[l]; c->st[l] = st[l];
        c->cr[l] = pi15 * wt[l] * s5;
        c->cn[l] = pi15 * wt[l] * s5 * st[l] * st[l];
        c->st2q[l] = st[l] * st[l] * 0.25;
    }
    /* |m_a| <= R |column a of h| holds the ellipsoid |h^{-T} m| <= R */
    const double R = 2.0 * sqrt(46.0) / st[0] / (2.0 * ORC_PI);
    const double len[3] = {fabs(h[0]), sqrt(h[1] * h[1] + h[4] * h[4]),
                           sqrt(h[2] * h[2] + h[5] * h[5] + h[8] * h[8])};
    for (int a = 0; a < 3; ++a) c->mm[a] = (int)ceil(R * len[a]) + 2;
    c->nx = 2 * c->mm[0] + 1; c->ny = 2 * c->mm[1] + 1; c->nz = 2 * c->mm[2] + 1;
    c->Gx = (double *)calloc((size_t)M * 3 * c->nx, sizeof(double));
    c->Gy = (double *)calloc((size_t)M * 3 * c->nx * c->ny, sizeof(double));
    for (int l = 0; l < M; ++l) {
        double s4 = 0.0;
        for (int i = 0; i < c->nx; ++i) {
            double gx[3] = {0, 0, 0};
            for (int j = 0; j < c->ny; ++j) {
                double g[3] = {0, 0, 0};
                for (int kz = 0; kz < c->nz; ++kz) {
                    int m[3] = {i - c->mm[0], j - c->mm[1], kz - c->mm[2]};
                    double k[3];
                    kvec_h(h, m, k);
                    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                    double e = exp(-(c->st2q[l] * k2));
                    for (int a = 0; a < 3; ++a) g[a] += k[a] * k[a] * e;
                    s4 += (k2 * k2) * e;
                }
                for (int a = 0; a < 3; ++a) {
                    c->Gy[(((size_t)l * 3 + a) * c->nx + i) * c->ny + j] = g[a];
                    gx[a] += g[a];
                }
            }
            for (int a = 0; a < 3; ++a) c->Gx[((size_t)l * 3 + a) * c->nx + i] = gx[a];
        }
        for (int a = 0; a < 3; ++a) {
            double sa = 0.0;
            for (int i = 0; i < c->nx; ++i) sa += c->Gx[((size_t)l * 3 + a) * c->nx + i];
            c->S[l][a] = sa;
        }
        c->Hr[l] = c->cr[l] * (c->S[l][0] + c->S[l][1] + c->S[l][2]);
        c->Hnr[l] = c->cn[l] * s4;
    }
    return c;
}

void orc_tri_free(tri_ctx *c)
{
    if (!c) return;
    free(c->Gx);
    free(c->Gy);
    free(c);
}

void orc_tri_normalizers(const tri_ctx *c, double *Hr, double *Hnr, int *mm)
{
    for (int l = 0; l < c->M; ++l) { Hr[l] = c->Hr[l]; Hnr[l] = c->Hnr[l]; }
    if (mm) for (int a = 0; a < 3; ++a) mm[a] = c->mm[a];
}

static void tri_targets(const tri_ctx *c, const int *m, double *pr, double *pnr)
{
    double k[3];
    kvec_h(c->h, m, k);
    double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    double a = 0, b = 0;
    for (int l = 0; l < c->M; ++l) {
        double e = exp(-(c->st2q[l] * k2));
        a += c->cr[l] * e;
        b += c->cn[l] * e;
    }
    *pr = k2 * a;
    *pnr = (k2 * k2) * b;
}

#define ORC_TRI_NQ 20

/* inverse CDF over m = 0, 1, -1, ... of a table indexed by m + mm */
static int walk_table(double target, const double *tab, int mm)
{
    double cum = 0.0;
    int last = 0;
    for (int k = 0; k <= 2 * mm; ++k) {
        int m = walk_index(k);
        cum += tab[m + mm];
        last = m;
        if (cum > target) return m;
    }
    return last;
}

static void tri_exact_draw_r(const tri_ctx *c, const uint64_t wds[4], int *m)
{
    double tot = 0;
    for (int l = 0; l < c->M; ++l) tot += c->Hr[l];
    double target = orc_u01(wds[0]) * tot, cum = 0;
    int lsel = c->M - 1, asel = 2, done = 0;
    for (int l = 0; l < c->M && !done; ++l)
        for (int a = 0; a < 3; ++a) {
            cum += c->cr[l] * c->S[l][a];
            if (cum > target) { lsel = l; asel = a; done = 1; break; }
        }
    const double *gx = c->Gx + ((size_t)lsel * 3 + asel) * c->nx;
    double tx = 0.0;
    for (int i = 0; i < c->nx; ++i) tx += gx[i];
    m[0] = walk_table(orc_u01(wds[1]) * tx, gx, c->mm[0]);
    const double *gy = c->Gy + (((size_t)lsel * 3 + asel) * c->nx + (m[0] + c->mm[0])) * c->ny;
    double ty = 0.0;
    for (int j = 0; j < c->ny; ++j) ty += gy[j];
    m[1] = walk_table(orc_u01(wds[2]) * ty, gy, c->mm[1]);
    /* m_2 given (m_0, m_1): weights k_a^2 e_l formed in walk order */
    double tz = 0.0;
    for (int kz = 0; kz < c->nz; ++kz) {
        int mm3[3] = {m[0], m[1], kz - c->mm[2]};
        double k[3];
        kvec_h(c->h, mm3, k);
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        tz += k[asel] * k[asel] * exp(-(c->st2q[lsel] * k2));
    }
    double target2 = orc_u01(wds[3]) * tz, cz = 0.0;
    int last = 0;
    m[2] = 0;
    for (int k = 0; k <= 2 * c->mm[2]; ++k) {
        int mm3[3] = {m[0], m[1], walk_index(k)};
        double kk[3];
        kvec_h(c->h, mm3, kk);
        double k2 = kk[0] * kk[0] + kk[1] * kk[1] + kk[2] * kk[2];
        cz += kk[asel] * kk[asel] * exp(-(c->st2q[lsel] * k2));
        last = mm3[2];
        if (cz > target2) break;
    }
    m[2] = last;
}

/* one exact draw from P^r (the chain's start state at index 0), for tests */
void orc_tri_draw_r(const tri_ctx *c, uint64_t seed, uint64_t sysid, uint64_t step, uint64_t index, int *m)
{
    uint64_t wds[4];
    draw4(seed, sysid, step, PUR_START, index, wds);
    tri_exact_draw_r(c, wds, m);
}

/* pr, pnr (unnormalised targets) and q (eq. proposal) of one mode */
void orc_tri_targets(const tri_ctx *c, const int *m, double *out)
{
    tri_targets(c, m, &out[0], &out[1]);
    out[2] = orc_tri_q(c->h, c->st[0], m, ORC_TRI_NQ);
}

/* the paper's construction (kind 0 of orc_sample_modes) for a general h */
void orc_tri_sample_modes(const tri_ctx *c, int P, uint64_t seed, uint64_t sysid, uint64_t step,
                          int *mr, int *mnr, double *stats)
{
    const double *h = c->h;
    const double sig_u = 1.0 / (sqrt(2.0) * ORC_PI * c->st[0]);
    uint64_t wds[4];
    int x[3];
    double pr, pnr;
    stats[0] = stats[1] = 0;
    draw4(seed, sysid, step, PUR_START, 0, wds);
    tri_exact_draw_r(c, wds, x);
    tri_targets(c, x, &pr, &pnr);
    double wcur = pr / orc_tri_q(h, c->st[0], x, ORC_TRI_NQ);
    for (int t = 1; t <= P; ++t) {
        double z[3], zz;
        draw4(seed, sysid, step, PUR_PROPOSAL, (uint64_t)(t - 1), wds);
        box_muller(wds[0], wds[1], &z[0], &z[1]);
        box_muller(wds[2], wds[3], &z[2], &zz);
        /* gamma = h^T (sigma_u z) */
        double g0 = h[0] * (z[0] * sig_u);
        double g1 = h[4] * (z[1] * sig_u) + h[1] * (z[0] * sig_u);
        double g2 = h[8] * (z[2] * sig_u) + (h[2] * (z[0] * sig_u) + h[5] * (z[1] * sig_u));
        int ms[3] = {(int)floor(g0 + 0.5), (int)floor(g1 + 0.5), (int)floor(g2 + 0.5)};
        double ws = 0.0;
        if (ms[0] || ms[1] || ms[2]) {
            tri_targets(c, ms, &pr, &pnr);
            ws = pr / orc_tri_q(h, c->st[0], ms, ORC_TRI_NQ);
        }
        draw4(seed, sysid, step, PUR_ACCEPT, (uint64_t)(t - 1), wds);
        if (orc_u01(wds[0]) * wcur < ws) {
            x[0] = ms[0]; x[1] = ms[1]; x[2] = ms[2];
            wcur = ws;
            stats[0] += 1;
        }
        mr[3 * (t - 1)] = x[0]; mr[3 * (t - 1) + 1] = x[1]; mr[3 * (t - 1) + 2] = x[2];
    }
    int y[3] = {mr[0], mr[1], mr[2]};
    tri_targets(c, y, &pr, &pnr);
    double gcur = pnr / pr;
    for (int t = 1; t <= P; ++t) {
        const int *xt = mr + 3 * (t - 1);
        tri_targets(c, xt, &pr, &pnr);
        double gt = pnr / pr;
        draw4(seed, sysid, step, PUR_ACCEPT, (uint64_t)(t - 1), wds);
        if (orc_u01(wds[1]) * gcur < gt) {
            y[0] = xt[0]; y[1] = xt[1]; y[2] = xt[2];
            gcur = gt;
            stats[1] += 1;
        }
        mnr[3 * (t - 1)] = y[0]; mnr[3 * (t - 1) + 1] = y[1]; mnr[3 * (t - 1) + 2] = y[2];
    }
}

/* eq. rho_k with k = 2 pi h^{-T} m */
void orc_rho_h(int N, const double *r, const double *q, const double *h, int nD, const int *D, double *rho)
{
#pragma omp parallel for schedule(static)
    for (int d = 0; d < nD; ++d) {
        double k[3];
        kvec_h(h, D + 3 * d, k);
        double re = 0, im = 0;
        for (int j = 0; j < N; ++j) {
            double th = k[0] * r[3 * j] + k[1] * r[3 * j + 1] + k[2] * r[3 * j + 2];
            re += q[j] * cos(th);
            im += q[j] * sin(th);
        }
        rho[2 * d] = re;
        rho[2 * d + 1] = im;
    }
}

/* orc_rb_longrange with k = 2 pi h^{-T} m and V = det h */
void orc_rb_longrange_h(int N, const double *r, const double *q, const double *h,
                        int P, int nD, const int *D, const int *cr, const int *cnr,
                        double Sr, double Snr, double ke, double *F, double *out,
                        double *Wr, double *Wnr, double *rho)
{
    const double V = fabs(det3(h));
    orc_rho_h(N, r, q, h, nD, D, rho);
    double Ar = 0, B[9] = {0};
    for (int d = 0; d < nD; ++d) {
        double k[3];
        kvec_h(h, D + 3 * d, k);
        double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
        double r2 = rho[2 * d] * rho[2 * d] + rho[2 * d + 1] * rho[2 * d + 1];
        Ar += cr[d] * r2 / k2;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) B[3 * a + b] += cnr[d] * r2 * k[a] * k[b] / (k2 * k2);
    }
    out[0] = ke * Sr / (4.0 * V * P) * Ar;
    for (int a = 0; a < 9; ++a) {
        Wr[a] = (a % 4 == 0) ? ke * Sr / (4.0 * V * P) * Ar : 0.0;
        Wnr[a] = -ke * Snr / (8.0 * V * P) * B[a];
    }
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        double f[3] = {0, 0, 0};
        for (int d = 0; d < nD; ++d) {
            if (!cr[d]) continue;
            double k[3];
            kvec_h(h, D + 3 * d, k);
            double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            double th = k[0] * r[3 * i] + k[1] * r[3 * i + 1] + k[2] * r[3 * i + 2];
            double g = rho[2 * d + 1] * cos(th) - rho[2 * d] * sin(th);
            for (int a = 0; a < 3; ++a) f[a] += cr[d] * k[a] * g / k2;
        }
        double cc = -ke * (0.5 * Sr) / P * q[i] / V;
        for (int a = 0; a < 3; ++a) F[3 * i + a] += cc * f[a];
    }
}

/* orc_force_eval for a general (upper-triangular) cell h, the paper's
 * sampler (kind 0) with the sums of tc (made for the same h and split);
 * outputs as orc_force_eval. */
void orc_force_eval_h(const orc_params *pp, const orc_system *sy, const double *r, const double *h,
                      const tri_ctx *tc, uint64_t step, double *F, double *en, double *W,
                      double *Wparts, int *modes_out)
{
    int N = sy->N, M = pp->M, ME = pp->ME, P = pp->P;
    int MM = M > ME ? M : ME;
    double *w = (double *)malloc(sizeof(double) * 4 * MM);
    double *s = w + MM, *wt = w + 2 * MM, *st = w + 3 * MM;
    orc_sog_terms(pp->b, pp->sigma, pp->omega, MM, w, s, wt, st);
    memset(F, 0, sizeof(double) * 3 * N);
    double esr[2], Wc[9], Wl[9];
    orc_short_range(N, r, sy->q, sy->type, sy->mol, h, pp->rc, M, wt, st, ME, w, s,
                    sy->ntypes, sy->lj_eps, sy->lj_sig, pp->ke, F, esr, Wc, Wl);
    int *mr = (int *)malloc(sizeof(int) * 6 * P);
    int *mnr = mr + 3 * P;
    double stats[2];
    orc_tri_sample_modes(tc, P, pp->seed, pp->sysid, step, mr, mnr, stats);
    if (modes_out) memcpy(modes_out, mr, sizeof(int) * 6 * P);
    int *D = (int *)malloc(sizeof(int) * 3 * 2 * P);
    int *cr = (int *)malloc(sizeof(int) * 2 * P), *cnr = (int *)malloc(sizeof(int) * 2 * P);
    int nD = orc_distinct(P, mr, P, mnr, D, cr, cnr);
    double Sr = 0, Snr = 0;
    for (int l = 0; l < M; ++l) { Sr += tc->Hr[l]; Snr += tc->Hnr[l]; }
    double *rho = (double *)malloc(sizeof(double) * 2 * nD);
    double uf, Wr[9], Wnr[9];
    orc_rb_longrange_h(N, r, sy->q, h, P, nD, D, cr, cnr, Sr, Snr, pp->ke, F, &uf, Wr, Wnr, rho);
    double ux, Wx[9], eb[2], Wb[9];
    orc_exclusions(sy->ne, sy->excl, r, sy->q, h, M, wt, st, ME, w, s, pp->ke, F, &ux, Wx);
    orc_bonded(sy->nb, sy->bonds, sy->bk, sy->br0, sy->na, sy->angles, sy->ak, sy->at0, r, h, F, eb, Wb);
    double us = orc_self_energy(pp->b, pp->sigma, pp->omega, ME, N, sy->q, pp->ke);
    en[0] = esr[0]; en[1] = uf; en[2] = us; en[3] = ux; en[4] = esr[1]; en[5] = eb[0]; en[6] = eb[1];
    en[7] = esr[0] + uf - us + ux;
    en[8] = nD;
    for (int a = 0; a < 9; ++a) {
        W[a] = Wc[a] + Wr[a] + Wnr[a] + Wl[a] + Wx[a] + Wb[a];
        if (Wparts) {
            Wparts[a] = Wc[a]; Wparts[9 + a] = Wr[a]; Wparts[18 + a] = Wnr[a];
            Wparts[27 + a] = Wl[a]; Wparts[36 + a] = Wx[a] + Wb[a];
        }
    }
    free(rho); free(D); free(cr); free(cnr); free(mr); free(w);
}

/* Algorithm 1 step 8 with the cell held fixed (Langevin NVT in a general
 * cell): the BAOAB splitting of orc_npt_run without the box terms; atoms are
 * wrapped into the cell by whole cell vectors, r <- r - h floor(h^{-1} r). */
void orc_nvt_run_h(const orc_params *pp, const orc_system *sy, const orc_integ *ig, const tri_ctx *tc,
                   double *r, double *p, double *F, double *W, uint64_t step0, int nsteps,
                   double *en_out, double *K_out)
{
    int N = sy->N;
    const double *h = tc->h;
    double hi[9], mvv2e = 1.0 / ig->ftm2v, K[9];
    inv3(h, hi);
    double c = exp(-ig->gamma * ig->dt);
    for (int n = 1; n <= nsteps; ++n) {
        uint64_t step = step0 + (uint64_t)n;
        for (int i = 0; i < 3 * N; ++i) p[i] += 0.5 * ig->dt * F[i] * ig->ftm2v;
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) r[3 * i + a] = r[3 * i + a] + p[3 * i + a] / sy->mass[i] * (0.5 * ig->dt);
        uint64_t wds[4];
        for (int i = 0; i < N; ++i) {
            double z[4];
            draw4(pp->seed, pp->sysid, step, PUR_ATOM, (uint64_t)i, wds);
            box_muller(wds[0], wds[1], &z[0], &z[1]);
            box_muller(wds[2], wds[3], &z[2], &z[3]);
            double sdv = sqrt((1.0 - c * c) * sy->mass[i] * ig->kB * ig->T * ig->ftm2v);
            for (int a = 0; a < 3; ++a) p[3 * i + a] = c * p[3 * i + a] + sdv * z[a];
        }
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < 3; ++a) r[3 * i + a] = r[3 * i + a] + p[3 * i + a] / sy->mass[i] * (0.5 * ig->dt);
        for (int i = 0; i < N; ++i) {
            double *x = r + 3 * i, f[3];
            for (int a = 0; a < 3; ++a) f[a] = floor(hi[3 * a] * x[0] + hi[3 * a + 1] * x[1] + hi[3 * a + 2] * x[2]);
            for (int a = 0; a < 3; ++a) x[a] -= h[3 * a] * f[0] + h[3 * a + 1] * f[1] + h[3 * a + 2] * f[2];
        }
        orc_force_eval_h(pp, sy, r, h, tc, step, F, en_out, W, NULL, NULL);
        for (int i = 0; i < 3 * N; ++i) p[i] += 0.5 * ig->dt * F[i] * ig->ftm2v;
    }
    kinetic(N, p, sy->mass, mvv2e, K);
    for (int a = 0; a < 9; ++a) K_out[a] = K[a];
}
