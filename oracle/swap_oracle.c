/*
 * swap_oracle.c -- plain FP64 CPU oracle for the associative bond-swap
 * potential (Ciarella & Ellenbroek, "Associative bond swaps in molecular
 * dynamics").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark use it.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What it computes (section "The swap potential"):
 *   U = sum_{i<j} u2(r_ij) + sum_i sum_{j<k in R(i)} a_ij a_ik vh(r_ij) vh(r_ik)
 *   - u2 for a reactive ("swap") type pair is the generalised Lennard-Jones
 *     v(r) = 4 eps [(sigma/r)^(2n) - (sigma/r)^n] of Eq. 2b, r < r_cut;
 *   - u2 for a "wca" type pair is the same form cut at its minimum
 *     r_min = sigma 2^(1/n) and shifted up by eps (purely repulsive; the
 *     paper's A-A and B-B interaction, section "Effect of swaps", n = 6);
 *   - vh is the normalised two-body term of Eq. pot: 1 for r <= r_min,
 *     -v(r)/eps beyond, 0 at and beyond r_cut;
 *   - the three-body term is Eq. 3bp with centre i and the unordered pair
 *     {j,k} of reactive partners of i; the prefactor lambda*eps of Eq. 3bp is
 *     written a_ij a_ik with a = sqrt(lambda eps) so that it factorises when
 *     the two pairs have different coefficients (reduces to lambda*eps for a
 *     single reactive type pair).
 *   - forces are -dU/dx by analytic differentiation of every pair and every
 *     triplet term separately; the triplet loop is explicit, O(n_r^2) per
 *     centre, exactly as Eq. 3bp is written (no per-centre partial sums);
 *   - the virial is W_ab = -sum over pair vectors r_ij (= x_i - x_j) of
 *     (r_ij)_a dU/d(r_ij)_b, which for the triplets is the content of Eq. p3.
 *
 * Optional harmonic bonds (orc_bonds): u = k/2 (r - r0)^2 for listed pairs,
 * minimum image, no cut-off, no exclusion of the bonded pair's own pair term.
 *
 * Optional "shifted" form of a swap pair (off by default, the paper's literal
 * form is unshifted): v_s = v - v(r_cut) and vh_s = (v(r_cut) - v)/(eps +
 * v(r_cut)) beyond r_min, continuous at r_cut and still equal to 1 at r_min.
 *
 * Decisions that turn a distance into an integer (is a pair inside its
 * cut-off, inside the neighbour-list radius, inside the bond radius) can be
 * taken in FP32 (fp32 = 1), on 32-bit fractions of the box edges:
 *   - each box edge is rounded to float, then to the 2^-48 grid: Lq =
 *     round(L 2^48) (halves away from zero), L' = Lq 2^-48;
 *   - a coordinate x is wrapped and put on the same grid: k = floor(x / L'),
 *     q = round-half-even((x - k L') 2^48), then q -= Lq if q >= Lq and
 *     q += Lq if q < 0;
 *   - its fraction is u = floor(q f / 2^64) with f = floor(2^96 / Lq);
 *   - a displacement component is the difference u_j - u_i taken modulo
 *     2^32 as a signed 32-bit integer (this is the minimum image), converted
 *     to float and multiplied by the float of Lq 2^-80 (the edge per 2^32);
 *   - d2 = (dx*dx + dy*dy) + dz*dz in IEEE float, one rounding per
 *     operation, no contraction (build with -ffp-contract=off), compared with
 *     the float of (cut*cut computed in double).
 * The values of the potential are always evaluated in FP64 from the double
 * displacement.
 *
 * Integrators: velocity Verlet (NVE) and BAOAB Langevin (NVT), Leimkuhler &
 * Matthews (2013).  The Langevin noise uses Philox4x32-10 (Salmon, Moraes,
 * Dror & Shaw, SC'11) written here from its published definition, mapped to
 * normals by the Box-Muller transform.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Built as is (gcc, no -fopenmp), every loop runs on one thread in the order
 * written.  Built a second time with -fopenmp (the benchmark's all-cores CPU
 * baseline only), the pair search splits the particles, and the force sums
 * split the pairs and the centres, over the threads in contiguous ranges;
 * each thread sums into its own buffers, added up in thread order.  The
 * terms are the same; only the order of the additions differs. */

#define ORC_KIND_NONE 0
#define ORC_KIND_WCA 1
#define ORC_KIND_SWAP 2

typedef struct {
    int kind;      /* ORC_KIND_* */
    int n;         /* exponent n of Eq. 2b (integer >= 1) */
    int shift;     /* swap pairs: 0 = literal Eq. 2b, 1 = shifted form */
    int pad;
    double eps;
    double sigma;
    double lambda3; /* lambda of Eq. 3bp */
    double rcut;    /* swap pairs: r_cut of Eq. 2b; wca pairs: ignored (r_min) */
    double rbond;   /* swap pairs: a reactive pair closer than this is a bond */
} orc_pair;

/* ---------------------------------------------------------------------- */
/* Eq. 2b and its derivatives, plain pow().                                */

static double lj_v(double r, double eps, double sigma, int n)
{
    double x = pow(sigma / r, (double)n);
    return 4.0 * eps * (x * x - x);
}

/* dv/dr */
static double lj_dv(double r, double eps, double sigma, int n)
{
    double x = pow(sigma / r, (double)n);
    return 4.0 * eps * (-2.0 * n * x * x + n * x) / r;
}

/* d2v/dr2 */
static double lj_d2v(double r, double eps, double sigma, int n)
{
    double x = pow(sigma / r, (double)n);
    return 4.0 * eps * (2.0 * n * (2.0 * n + 1.0) * x * x - n * (n + 1.0) * x) / (r * r);
}

double orc_v2(double r, double eps, double sigma, int n) { return lj_v(r, eps, sigma, n); }
double orc_dv2(double r, double eps, double sigma, int n) { return lj_dv(r, eps, sigma, n); }

static double pair_rmin(const orc_pair *p) { return p->sigma * pow(2.0, 1.0 / p->n); }

/* Two-body energy u2(r) and its first two derivatives for one pair type, for
 * a pair already decided to be inside its cut-off (the decision is taken by
 * the caller, in the decision precision; a WCA pair is inside for r < r_min,
 * where u2 and du2/dr go to zero continuously). */
static void pair_u2(const orc_pair *p, double r, double *u, double *du, double *d2u)
{
    *u = *du = *d2u = 0.0;
    if (p->kind == ORC_KIND_WCA) {
        *u = lj_v(r, p->eps, p->sigma, p->n) + p->eps;
        *du = lj_dv(r, p->eps, p->sigma, p->n);
        *d2u = lj_d2v(r, p->eps, p->sigma, p->n);
    } else if (p->kind == ORC_KIND_SWAP) {
        double vc = p->shift ? lj_v(p->rcut, p->eps, p->sigma, p->n) : 0.0;
        *u = lj_v(r, p->eps, p->sigma, p->n) - vc;
        *du = lj_dv(r, p->eps, p->sigma, p->n);
        *d2u = lj_d2v(r, p->eps, p->sigma, p->n);
    }
}

/* Eq. pot: the normalised two-body term vh(r) and its derivatives, for a
 * swap pair already decided to be inside r_cut. */
static void pair_vhat(const orc_pair *p, double r, double *vh, double *dvh, double *d2vh)
{
    *vh = *dvh = *d2vh = 0.0;
    if (p->kind != ORC_KIND_SWAP)
        return;
    if (r <= pair_rmin(p)) {
        *vh = 1.0;
        return;
    }
    double vc = p->shift ? lj_v(p->rcut, p->eps, p->sigma, p->n) : 0.0;
    double den = p->eps + vc;
    *vh = (vc - lj_v(r, p->eps, p->sigma, p->n)) / den;
    *dvh = -lj_dv(r, p->eps, p->sigma, p->n) / den;
    *d2vh = -lj_d2v(r, p->eps, p->sigma, p->n) / den;
}

/* Eq. pot with its cut-off applied (vh = 0 for r >= r_cut). */
double orc_vhat(const orc_pair *p, double r)
{
    double a, b, c;
    if (p->kind != ORC_KIND_SWAP || r >= p->rcut)
        return 0.0;
    pair_vhat(p, r, &a, &b, &c);
    return a;
}

/* Two-body energy with its cut-off applied. */
double orc_u2(const orc_pair *p, double r)
{
    double a, b, c;
    if (p->kind == ORC_KIND_WCA && r >= p->sigma * pow(2.0, 1.0 / p->n))
        return 0.0;
    if (p->kind == ORC_KIND_SWAP && r >= p->rcut)
        return 0.0;
    if (p->kind == ORC_KIND_NONE)
        return 0.0;
    pair_u2(p, r, &a, &b, &c);
    return a;
}

/* ---------------------------------------------------------------------- */
/* Distance decisions.                                                     */

static double wrap_d(double d, double L)
{
    if (d > 0.5 * L)
        return d - L;
    if (d < -0.5 * L)
        return d + L;
    return d;
}

/* What the decisions of one call need: the positions and box, and in FP32
 * the box fractions of every coordinate (computed once). */
typedef struct {
    const double *x, *box;
    int fp32;
    uint32_t *u; /* [3n] */
    float s[3];  /* float of Lq 2^-80 */
} decider;

/* 32-bit fraction of coordinate x along an edge of Lq grid units (the rule
 * in the header). */
static uint32_t box_fraction(double x, long long Lq, uint64_t f)
{
    double L = (double)Lq * 0x1p-48;
    double k = floor(x / L);
    double xw = x - k * L;
    long long q = llrint(xw * 0x1p48);
    if (q >= Lq)
        q -= Lq;
    if (q < 0)
        q += Lq;
    return (uint32_t)(((unsigned __int128)(uint64_t)q * f) >> 64);
}

static int decider_init(decider *dc, int n, const double *x, const double *box, int fp32)
{
    dc->x = x;
    dc->box = box;
    dc->fp32 = fp32;
    dc->u = NULL;
    if (!fp32)
        return 0;
    dc->u = (uint32_t *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(uint32_t));
    if (!dc->u)
        return -1;
    for (int c = 0; c < 3; c++) {
        long long Lq = llround((double)(float)box[c] * 0x1p48);
        uint64_t f = (uint64_t)(((unsigned __int128)1 << 96) / (unsigned __int128)Lq);
        dc->s[c] = (float)((double)Lq * 0x1p-80);
        for (int i = 0; i < n; i++)
            dc->u[3 * i + c] = box_fraction(x[3 * i + c], Lq, f);
    }
    return 0;
}

static void decider_free(decider *dc)
{
    free(dc->u);
    dc->u = NULL;
}

/* Squared minimum-image distance of particles i and j used for integer
 * decisions. */
static double decision_d2(const decider *dc, int i, int j)
{
    if (dc->fp32) {
        float d[3];
        for (int c = 0; c < 3; c++) {
            int32_t du = (int32_t)(dc->u[3 * j + c] - dc->u[3 * i + c]);
            d[c] = (float)du * dc->s[c];
        }
        float s = d[0] * d[0];
        float t = d[1] * d[1];
        s = s + t;
        t = d[2] * d[2];
        s = s + t;
        return (double)s;
    }
    const double *xi = &dc->x[3 * i], *xj = &dc->x[3 * j], *box = dc->box;
    double dx = wrap_d(xj[0] - xi[0], box[0]);
    double dy = wrap_d(xj[1] - xi[1], box[1]);
    double dz = wrap_d(xj[2] - xi[2], box[2]);
    double s = dx * dx;
    double t = dy * dy;
    s = s + t;
    t = dz * dz;
    s = s + t;
    return s;
}

/* The squared threshold a decision compares against, in the same precision. */
static double decision_cut2(double cut, int fp32)
{
    double c2 = cut * cut;
    return fp32 ? (double)(float)c2 : c2;
}

/* Interaction cut-off of a pair type (0 when the pair does not interact). */
static double pair_rcut(const orc_pair *p)
{
    if (p->kind == ORC_KIND_WCA)
        return pair_rmin(p);
    if (p->kind == ORC_KIND_SWAP)
        return p->rcut;
    return 0.0;
}

/* ---------------------------------------------------------------------- */
/* Candidate pairs from a plain linked-cell list (or all pairs for boxes   */
/* too small for a 3x3x3 stencil).                                         */

typedef struct {
    int i, j;
} ipair;

typedef struct {
    ipair *a;
    long n, cap;
} pairvec;

static int pv_push(pairvec *v, int i, int j)
{
    if (v->n == v->cap) {
        long nc = v->cap ? 2 * v->cap : 1024;
        ipair *na = (ipair *)realloc(v->a, (size_t)nc * sizeof(ipair));
        if (!na)
            return -1;
        v->a = na;
        v->cap = nc;
    }
    v->a[v->n].i = i;
    v->a[v->n].j = j;
    v->n++;
    return 0;
}

/* The pairs (i, j > i) of particle i from the 27 cells around its own,
 * appended to out.  Returns 0 or -1 (memory). */
static int cell_pairs(int i, const int *type, int ntypes, const orc_pair *tab, const decider *dc, double extra,
                      int fp32, const int nc[3], const int *head, const int *next, const int *cid, pairvec *out)
{
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int cx = (cid[3 * i] + dx + nc[0]) % nc[0];
                int cy = (cid[3 * i + 1] + dy + nc[1]) % nc[1];
                int cz = (cid[3 * i + 2] + dz + nc[2]) % nc[2];
                long c = ((long)cz * nc[1] + cy) * nc[0] + cx;
                for (int j = head[c]; j >= 0; j = next[j]) {
                    if (j <= i)
                        continue;
                    const orc_pair *p = &tab[type[i] * ntypes + type[j]];
                    double cut = pair_rcut(p);
                    if (cut <= 0.0)
                        continue;
                    if (decision_d2(dc, i, j) < decision_cut2(cut + extra, fp32))
                        if (pv_push(out, i, j))
                            return -1;
                }
            }
    return 0;
}

/* All unordered pairs i<j whose squared decision distance is below the
 * pair type's cut2 (cut = pair cut-off + extra).  Returns 0 or -1 (memory). */
static int find_pairs(int n, const double *x, const int *type, int ntypes, const orc_pair *tab,
                      const double *box, const decider *dc, double extra, pairvec *out)
{
    const int fp32 = dc->fp32;
    double cmax = 0.0;
    for (int t = 0; t < ntypes * ntypes; t++) {
        double c = pair_rcut(&tab[t]);
        if (c > 0.0 && c + extra > cmax)
            cmax = c + extra;
    }
    out->n = 0;
    if (cmax <= 0.0 || n < 2)
        return 0;
    int nc[3];
    for (int d = 0; d < 3; d++) {
        nc[d] = (int)floor(box[d] / cmax);
        if (nc[d] < 1)
            nc[d] = 1;
    }
    int brute = (nc[0] < 3 || nc[1] < 3 || nc[2] < 3);
    if (brute) {
        for (int i = 0; i < n; i++)
            for (int j = i + 1; j < n; j++) {
                const orc_pair *p = &tab[type[i] * ntypes + type[j]];
                double c = pair_rcut(p);
                if (c <= 0.0)
                    continue;
                if (decision_d2(dc, i, j) < decision_cut2(c + extra, fp32))
                    if (pv_push(out, i, j))
                        return -1;
            }
        return 0;
    }
    long ncell = (long)nc[0] * nc[1] * nc[2];
    int *head = (int *)malloc((size_t)ncell * sizeof(int));
    int *next = (int *)malloc((size_t)n * sizeof(int));
    int *cid = (int *)malloc((size_t)n * 3 * sizeof(int));
    if (!head || !next || !cid) {
        free(head);
        free(next);
        free(cid);
        return -1;
    }
    for (long c = 0; c < ncell; c++)
        head[c] = -1;
    for (int i = 0; i < n; i++) {
        int c3[3];
        for (int d = 0; d < 3; d++) {
            double s = x[3 * i + d] / box[d];
            s -= floor(s);
            int k = (int)(s * nc[d]);
            if (k >= nc[d])
                k = nc[d] - 1;
            if (k < 0)
                k = 0;
            c3[d] = k;
            cid[3 * i + d] = k;
        }
        long c = ((long)c3[2] * nc[1] + c3[1]) * nc[0] + c3[0];
        next[i] = head[c];
        head[c] = i;
    }
    int err = 0;
#ifdef _OPENMP
    int nt = omp_get_max_threads();
    pairvec *tv = (pairvec *)calloc((size_t)nt, sizeof(pairvec));
    if (!tv)
        err = 1;
    else {
#pragma omp parallel num_threads(nt) reduction(| : err)
        {
            pairvec *mine = &tv[omp_get_thread_num()];
#pragma omp for schedule(static)
            for (int i = 0; i < n; i++)
                err |= cell_pairs(i, type, ntypes, tab, dc, extra, fp32, nc, head, next, cid, mine);
        }
        /* contiguous ranges in thread order: the serial order of the pairs */
        for (int t = 0; t < nt && !err; t++)
            for (long q = 0; q < tv[t].n && !err; q++)
                err |= pv_push(out, tv[t].a[q].i, tv[t].a[q].j);
        for (int t = 0; t < nt; t++)
            free(tv[t].a);
        free(tv);
    }
#else
    for (int i = 0; i < n && !err; i++)
        err = cell_pairs(i, type, ntypes, tab, dc, extra, fp32, nc, head, next, cid, out);
#endif
    free(head);
    free(next);
    free(cid);
    return err ? -1 : 0;
}

/* ---------------------------------------------------------------------- */
/* Energy, forces, virial.                                                 */

/* out[0] = U2, out[1] = U3, out[2..7] = W (xx, yy, zz, xy, xz, yz),
 * out[8] = number of bonds.
 * scales (may be NULL): [0] energy scale of U2, [1] of U3, [2] virial scale.
 * fscale (may be NULL): per-particle force scale, the sum over every term
 * acting on the particle of |term| + r |d term/dr| (first-order sensitivity
 * of the term to a relative perturbation of its distances).
 * force (may be NULL): 3n doubles. */
/* Sums accumulated over the terms of one evaluation. */
typedef struct {
    double U2, U3, W[6], sU2, sU3, sW;
    long nb;
} orc_sums;

/* The two-body terms of the pair (i, j): energy, forces, virial, error
 * scales and bond count, added to s, force (may be NULL) and fscale (may be
 * NULL). */
static void pair_terms(int i, int j, const double *x, const int *type, int ntypes, const orc_pair *tab,
                       const double *box, const decider *dc, int fp32, orc_sums *s, double *force,
                       double *fscale)
{
    const orc_pair *p = &tab[type[i] * ntypes + type[j]];
    double d[3];
    for (int c = 0; c < 3; c++)
        d[c] = wrap_d(x[3 * i + c] - x[3 * j + c], box[c]); /* r_ij = x_i - x_j */
    double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double u, du, d2u;
    pair_u2(p, r, &u, &du, &d2u);
    s->U2 += u;
    s->sU2 += fabs(u) + r * fabs(du);
    /* F_i = -du/dr * d/r ; F_j = -F_i */
    double g = -du / r;
    if (force)
        for (int c = 0; c < 3; c++) {
            force[3 * i + c] += g * d[c];
            force[3 * j + c] -= g * d[c];
        }
    s->W[0] += g * d[0] * d[0];
    s->W[1] += g * d[1] * d[1];
    s->W[2] += g * d[2] * d[2];
    s->W[3] += g * d[0] * d[1];
    s->W[4] += g * d[0] * d[2];
    s->W[5] += g * d[1] * d[2];
    s->sW += r * fabs(du) + r * r * fabs(d2u);
    if (fscale) {
        double sc = fabs(du) + r * fabs(d2u);
        fscale[i] += sc;
        fscale[j] += sc;
    }
    if (p->kind == ORC_KIND_SWAP && decision_d2(dc, i, j) < decision_cut2(p->rbond, fp32))
        s->nb++;
}

/* Eq. 3bp for centre i: every unordered pair {j, k} of its reactive partners
 * rpart[rstart[i] .. rstart[i + 1]), one explicit term each, added to s,
 * force (may be NULL) and fscale (may be NULL). */
static void centre_terms(int i, const long *rstart, const int *rpart, const double *x, const int *type,
                         int ntypes, const orc_pair *tab, const double *box, orc_sums *s, double *force,
                         double *fscale)
{
    for (long qa = rstart[i]; qa < rstart[i + 1]; qa++) {
        for (long qb = qa + 1; qb < rstart[i + 1]; qb++) {
            int j = rpart[qa], k = rpart[qb];
            const orc_pair *pj = &tab[type[i] * ntypes + type[j]];
            const orc_pair *pk = &tab[type[i] * ntypes + type[k]];
            double dj[3], dk[3];
            for (int c = 0; c < 3; c++) {
                dj[c] = wrap_d(x[3 * i + c] - x[3 * j + c], box[c]);
                dk[c] = wrap_d(x[3 * i + c] - x[3 * k + c], box[c]);
            }
            double rj = sqrt(dj[0] * dj[0] + dj[1] * dj[1] + dj[2] * dj[2]);
            double rk = sqrt(dk[0] * dk[0] + dk[1] * dk[1] + dk[2] * dk[2]);
            double hj, dhj, d2hj, hk, dhk, d2hk;
            pair_vhat(pj, rj, &hj, &dhj, &d2hj);
            pair_vhat(pk, rk, &hk, &dhk, &d2hk);
            double aj = sqrt(pj->lambda3 * pj->eps);
            double ak = sqrt(pk->lambda3 * pk->eps);
            double pref = aj * ak;
            double v3 = pref * hj * hk;
            s->U3 += v3;
            s->sU3 += pref * (fabs(hj * hk) + rj * fabs(dhj * hk) + rk * fabs(hj * dhk));
            /* dU/drj = pref dhj hk ; dU/drk = pref hj dhk */
            double dUj = pref * dhj * hk;
            double dUk = pref * hj * dhk;
            double gj = -dUj / rj; /* force on i from the (i,j) leg: gj * dj */
            double gk = -dUk / rk;
            if (force)
                for (int c = 0; c < 3; c++) {
                    force[3 * i + c] += gj * dj[c] + gk * dk[c];
                    force[3 * j + c] -= gj * dj[c];
                    force[3 * k + c] -= gk * dk[c];
                }
            s->W[0] += gj * dj[0] * dj[0] + gk * dk[0] * dk[0];
            s->W[1] += gj * dj[1] * dj[1] + gk * dk[1] * dk[1];
            s->W[2] += gj * dj[2] * dj[2] + gk * dk[2] * dk[2];
            s->W[3] += gj * dj[0] * dj[1] + gk * dk[0] * dk[1];
            s->W[4] += gj * dj[0] * dj[2] + gk * dk[0] * dk[2];
            s->W[5] += gj * dj[1] * dj[2] + gk * dk[1] * dk[2];
            double sj = pref * (fabs(dhj * hk) + rj * fabs(d2hj * hk) + rk * fabs(dhj * dhk));
            double sk = pref * (fabs(hj * dhk) + rk * fabs(hj * d2hk) + rj * fabs(dhj * dhk));
            s->sW += rj * sj + rk * sk;
            if (fscale) {
                fscale[i] += sj + sk;
                fscale[j] += sj;
                fscale[k] += sk;
            }
        }
    }
}

#ifdef _OPENMP
/* The pair terms (what = 0, count = pairs) or the centre terms (what = 1,
 * count = n) on every thread, each over a contiguous range into its own sums
 * and buffers, then added to s, force and fscale in thread order. */
static int threaded_terms(int what, long count, const pairvec *pv, const long *rstart, const int *rpart, int n,
                          const double *x, const int *type, int ntypes, const orc_pair *tab, const double *box,
                          const decider *dc, int fp32, orc_sums *s, double *force, double *fscale)
{
    int nt = omp_get_max_threads();
    orc_sums *ts = (orc_sums *)calloc((size_t)nt, sizeof(orc_sums));
    double *fb = force ? (double *)calloc((size_t)nt * 3 * n, sizeof(double)) : NULL;
    double *sb = fscale ? (double *)calloc((size_t)nt * n, sizeof(double)) : NULL;
    if (!ts || (force && !fb) || (fscale && !sb)) {
        free(ts);
        free(fb);
        free(sb);
        return -1;
    }
#pragma omp parallel num_threads(nt)
    {
        int t = omp_get_thread_num();
        double *ft = fb ? fb + (size_t)t * 3 * n : NULL;
        double *st = sb ? sb + (size_t)t * n : NULL;
#pragma omp for schedule(static)
        for (long q = 0; q < count; q++) {
            if (what == 0)
                pair_terms(pv->a[q].i, pv->a[q].j, x, type, ntypes, tab, box, dc, fp32, &ts[t], ft, st);
            else
                centre_terms((int)q, rstart, rpart, x, type, ntypes, tab, box, &ts[t], ft, st);
        }
    }
    for (int t = 0; t < nt; t++) {
        s->U2 += ts[t].U2;
        s->U3 += ts[t].U3;
        for (int c = 0; c < 6; c++)
            s->W[c] += ts[t].W[c];
        s->sU2 += ts[t].sU2;
        s->sU3 += ts[t].sU3;
        s->sW += ts[t].sW;
        s->nb += ts[t].nb;
    }
    if (force)
        for (long k = 0; k < 3L * n; k++)
            for (int t = 0; t < nt; t++)
                force[k] += fb[(size_t)t * 3 * n + k];
    if (fscale)
        for (long k = 0; k < n; k++)
            for (int t = 0; t < nt; t++)
                fscale[k] += sb[(size_t)t * n + k];
    free(ts);
    free(fb);
    free(sb);
    return 0;
}
#endif

int orc_forces(int n, const double *x, const int *type, int ntypes, const orc_pair *tab,
               const double *box, int fp32, double *force, double *out, double *scales,
               double *fscale)
{
    pairvec pv = {0, 0, 0};
    decider dc;
    if (decider_init(&dc, n, x, box, fp32))
        return -1;
    if (find_pairs(n, x, type, ntypes, tab, box, &dc, 0.0, &pv)) {
        decider_free(&dc);
        return -1;
    }
    orc_sums sm;
    memset(&sm, 0, sizeof(sm));
    if (force)
        memset(force, 0, (size_t)n * 3 * sizeof(double));
    if (fscale)
        memset(fscale, 0, (size_t)n * sizeof(double));

    /* Per-centre lists of reactive partners (index into pv). */
    int *rcount = (int *)calloc((size_t)(n > 0 ? n : 1), sizeof(int));
    if (!rcount) {
        free(pv.a);
        decider_free(&dc);
        return -1;
    }

    /* Two-body terms, pair by pair. */
    int err = 0;
#ifdef _OPENMP
    err = threaded_terms(0, pv.n, &pv, NULL, NULL, n, x, type, ntypes, tab, box, &dc, fp32, &sm, force, fscale);
#else
    for (long q = 0; q < pv.n; q++)
        pair_terms(pv.a[q].i, pv.a[q].j, x, type, ntypes, tab, box, &dc, fp32, &sm, force, fscale);
#endif
    for (long q = 0; q < pv.n; q++) {
        int i = pv.a[q].i, j = pv.a[q].j;
        if (tab[type[i] * ntypes + type[j]].kind == ORC_KIND_SWAP) {
            rcount[i]++;
            rcount[j]++;
        }
    }

    /* CSR of reactive partners per centre. */
    long *rstart = (long *)malloc((size_t)(n + 1) * sizeof(long));
    long total = 0;
    for (int i = 0; i < n; i++)
        total += rcount[i];
    int *rpart = (int *)malloc((size_t)(total > 0 ? total : 1) * sizeof(int));
    if (err || !rstart || !rpart) {
        free(rstart);
        free(rpart);
        free(rcount);
        free(pv.a);
        decider_free(&dc);
        return -1;
    }
    rstart[0] = 0;
    for (int i = 0; i < n; i++)
        rstart[i + 1] = rstart[i] + rcount[i];
    for (int i = 0; i < n; i++)
        rcount[i] = 0;
    for (long q = 0; q < pv.n; q++) {
        int i = pv.a[q].i, j = pv.a[q].j;
        if (tab[type[i] * ntypes + type[j]].kind != ORC_KIND_SWAP)
            continue;
        rpart[rstart[i] + rcount[i]++] = j;
        rpart[rstart[j] + rcount[j]++] = i;
    }

    /* Eq. 3bp: explicit loop over every centre i and unordered {j,k}. */
#ifdef _OPENMP
    err = threaded_terms(1, n, NULL, rstart, rpart, n, x, type, ntypes, tab, box, &dc, fp32, &sm, force, fscale);
#else
    for (int i = 0; i < n; i++)
        centre_terms(i, rstart, rpart, x, type, ntypes, tab, box, &sm, force, fscale);
#endif

    out[0] = sm.U2;
    out[1] = sm.U3;
    for (int c = 0; c < 6; c++)
        out[2 + c] = sm.W[c];
    out[8] = (double)sm.nb;
    if (scales) {
        scales[0] = sm.sU2;
        scales[1] = sm.sU3;
        scales[2] = sm.sW;
    }
    free(rstart);
    free(rpart);
    free(rcount);
    free(pv.a);
    decider_free(&dc);
    return err ? -1 : 0;
}

/* Harmonic bonds of a fixed topology (the chains of the vitrimer network, a
 * NEXT item of this build; the paper's vitrimer section uses bonded chains
 * without giving a form): u = k/2 (r - r0)^2 for every listed pair (i, j),
 * minimum image, no cut-off.  ADDS the forces to force (3n, may be NULL) and
 * the scales to fscale (n, may be NULL); out[0] = bond energy, out[1..6] =
 * virial (xx yy zz xy xz yz, same convention as orc_forces); scale[0..1] =
 * energy and virial error scales (may be NULL). */
void orc_bonds(int n, const double *x, const double *box, long nb, const int *bonds, double k,
               double r0, double *force, double *out, double *fscale, double *scale)
{
    double U = 0.0, W[6] = {0, 0, 0, 0, 0, 0}, sU = 0.0, sW = 0.0;
    (void)n;
    for (long b = 0; b < nb; b++) {
        int i = bonds[2 * b], j = bonds[2 * b + 1];
        double d[3];
        for (int c = 0; c < 3; c++)
            d[c] = wrap_d(x[3 * i + c] - x[3 * j + c], box[c]); /* r_ij = x_i - x_j */
        double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double u = 0.5 * k * (r - r0) * (r - r0);
        double du = k * (r - r0), d2u = k;
        U += u;
        sU += fabs(u) + r * fabs(du);
        double g = -du / r;
        if (force)
            for (int c = 0; c < 3; c++) {
                force[3 * i + c] += g * d[c];
                force[3 * j + c] -= g * d[c];
            }
        W[0] += g * d[0] * d[0];
        W[1] += g * d[1] * d[1];
        W[2] += g * d[2] * d[2];
        W[3] += g * d[0] * d[1];
        W[4] += g * d[0] * d[2];
        W[5] += g * d[1] * d[2];
        sW += r * fabs(du) + r * r * fabs(d2u);
        if (fscale) {
            double sc = fabs(du) + r * fabs(d2u);
            fscale[i] += sc;
            fscale[j] += sc;
        }
    }
    out[0] = U;
    for (int c = 0; c < 6; c++)
        out[1 + c] = W[c];
    if (scale) {
        scale[0] = sU;
        scale[1] = sW;
    }
}

/* Neighbour-list membership: for every particle i, the sorted indices j != i
 * whose squared decision distance is below (r_cut(ti,tj) + skin)^2, for
 * interacting type pairs only.  counts[i] = number of such j; nbr is n*maxn
 * row-major.  Returns the largest count (rows longer than maxn are cut), or
 * -1 on allocation failure. */
int orc_nlist(int n, const double *x, const int *type, int ntypes, const orc_pair *tab,
              const double *box, int fp32, double skin, int maxn, int *counts, int *nbr)
{
    pairvec pv = {0, 0, 0};
    decider dc;
    if (decider_init(&dc, n, x, box, fp32))
        return -1;
    int rc = find_pairs(n, x, type, ntypes, tab, box, &dc, skin, &pv);
    decider_free(&dc);
    if (rc)
        return -1;
    for (int i = 0; i < n; i++)
        counts[i] = 0;
    for (long q = 0; q < pv.n; q++) {
        int i = pv.a[q].i, j = pv.a[q].j;
        if (counts[i] < maxn)
            nbr[(long)i * maxn + counts[i]] = j;
        counts[i]++;
        if (counts[j] < maxn)
            nbr[(long)j * maxn + counts[j]] = i;
        counts[j]++;
    }
    int mx = 0;
    for (int i = 0; i < n; i++) {
        int c = counts[i] < maxn ? counts[i] : maxn;
        int *row = &nbr[(long)i * maxn];
        for (int a = 1; a < c; a++) { /* insertion sort */
            int v = row[a], b = a - 1;
            while (b >= 0 && row[b] > v) {
                row[b + 1] = row[b];
                b--;
            }
            row[b + 1] = v;
        }
        if (counts[i] > mx)
            mx = counts[i];
    }
    free(pv.a);
    return mx;
}

/* A second per-particle force scale: over i's interacting pairs, |du2/dr|
 * (1 + lambda (S_i + S_j)) for a reactive pair (S_i: the sum of vh over i's
 * reactive partners inside r_cut) and |du2/dr| for the others -- the size of
 * the two-body forces, each amplified by the three-body factor it can
 * receive (Eq. 3bp through S_i).  Unlike the scale orc_forces returns it
 * has no term for the sensitivity to the distances, so it vanishes for a
 * particle whose pairs all sit at r_min.  Returns 0 or -1 (memory). */
int orc_fscale_c9(int n, const double *x, const int *type, int ntypes, const orc_pair *tab,
                  const double *box, int fp32, double *scale)
{
    pairvec pv = {0, 0, 0};
    decider dc;
    if (decider_init(&dc, n, x, box, fp32))
        return -1;
    if (find_pairs(n, x, type, ntypes, tab, box, &dc, 0.0, &pv)) {
        decider_free(&dc);
        return -1;
    }
    double *S = (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    if (!S) {
        free(pv.a);
        decider_free(&dc);
        return -1;
    }
    memset(scale, 0, (size_t)n * sizeof(double));
    for (int pass = 0; pass < 2; pass++)
        for (long q = 0; q < pv.n; q++) {
            int i = pv.a[q].i, j = pv.a[q].j;
            const orc_pair *p = &tab[type[i] * ntypes + type[j]];
            double d[3];
            for (int c = 0; c < 3; c++)
                d[c] = wrap_d(x[3 * i + c] - x[3 * j + c], box[c]);
            double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (pass == 0) {
                if (p->kind == ORC_KIND_SWAP) {
                    double vh, dvh, d2vh;
                    pair_vhat(p, r, &vh, &dvh, &d2vh);
                    S[i] += vh;
                    S[j] += vh;
                }
            } else {
                double u, du, d2u;
                pair_u2(p, r, &u, &du, &d2u);
                double w = fabs(du);
                if (p->kind == ORC_KIND_SWAP)
                    w *= 1.0 + p->lambda3 * (S[i] + S[j]);
                scale[i] += w;
                scale[j] += w;
            }
        }
    free(S);
    free(pv.a);
    decider_free(&dc);
    return 0;
}

/* Threads the force sums use (1 unless built with OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 and Box-Muller normals.                                   */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Three standard normals for (seed, step, tag, purpose): counter words are
 * (tag, step low, step high, purpose), key words (seed low, seed high);
 * u = (w + 0.5) 2^-32; z0, z1 from (u0, u1), z2 from (u2, u3). */
void orc_normals3(uint64_t seed, uint64_t step, uint32_t tag, uint32_t purpose, double z[3])
{
    uint32_t ctr[4] = {tag, (uint32_t)step, (uint32_t)(step >> 32), purpose};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    const double two_pi = 6.283185307179586476925286766559;
    double u0 = ((double)w[0] + 0.5) * 2.3283064365386962890625e-10;
    double u1 = ((double)w[1] + 0.5) * 2.3283064365386962890625e-10;
    double u2 = ((double)w[2] + 0.5) * 2.3283064365386962890625e-10;
    double u3 = ((double)w[3] + 0.5) * 2.3283064365386962890625e-10;
    double ra = sqrt(-2.0 * log(u0));
    double rb = sqrt(-2.0 * log(u2));
    z[0] = ra * cos(two_pi * u1);
    z[1] = ra * sin(two_pi * u1);
    z[2] = rb * cos(two_pi * u3);
}

/* ---------------------------------------------------------------------- */
/* Integrators.                                                            */

/* Advance nsteps from step index step0.  BAOAB when gamma > 0 (NVT), else
 * velocity Verlet (NVE).  x is kept wrapped into [0, L) with image counts in
 * img (3n ints, may be NULL).  thermo (may be NULL) receives per step
 * [U2, U3, K, W0..W5, n_bonds, U_bond] (11 doubles) after the step (W includes
 * the bonds' virial).  Langevin step k (advancing state step0+k) draws its
 * normals with step value step0+k and the particle's tag, purpose 1.  nb
 * harmonic bonds (orc_bonds; nb = 0: none) act besides the pair terms. */
static int run_forces(int n, const double *x, const int *type, int ntypes, const orc_pair *tab,
                      const double *box, int fp32, double *F, double *out, long nb, const int *bonds,
                      double kb, double r0)
{
    if (orc_forces(n, x, type, ntypes, tab, box, fp32, F, out, NULL, NULL))
        return -1;
    out[9] = 0.0;
    if (nb > 0) {
        double ob[7];
        orc_bonds(n, x, box, nb, bonds, kb, r0, F, ob, NULL, NULL);
        for (int c = 0; c < 6; c++)
            out[2 + c] += ob[1 + c];
        out[9] = ob[0];
    }
    return 0;
}

int orc_run(int n, double *x, double *v, int *img, const int *type, const double *mass,
            const uint32_t *tag, int ntypes, const orc_pair *tab, const double *box, int fp32,
            double dt, int nsteps, double kT, double gamma, uint64_t seed, uint64_t step0,
            double *thermo, long nb, const int *bonds, double kb, double r0)
{
    double *F = (double *)malloc((size_t)(n > 0 ? n : 1) * 3 * sizeof(double));
    double out[10];
    if (!F)
        return -1;
    if (run_forces(n, x, type, ntypes, tab, box, fp32, F, out, nb, bonds, kb, r0)) {
        free(F);
        return -1;
    }
    double c = exp(-gamma * dt);
    for (int s = 0; s < nsteps; s++) {
        for (int i = 0; i < n; i++) {
            double im = 1.0 / mass[i];
            for (int d = 0; d < 3; d++) {
                v[3 * i + d] += 0.5 * dt * F[3 * i + d] * im; /* B */
                x[3 * i + d] += 0.5 * dt * v[3 * i + d];      /* A */
            }
            if (gamma > 0.0) { /* O */
                double z[3];
                orc_normals3(seed, step0 + (uint64_t)s, tag[i], 1u, z);
                double sd = sqrt((1.0 - c * c) * kT * im);
                for (int d = 0; d < 3; d++)
                    v[3 * i + d] = c * v[3 * i + d] + sd * z[d];
            }
            for (int d = 0; d < 3; d++) {
                x[3 * i + d] += 0.5 * dt * v[3 * i + d]; /* A */
                double L = box[d];
                double k = floor(x[3 * i + d] / L);
                if (k != 0.0) {
                    x[3 * i + d] -= k * L;
                    if (x[3 * i + d] >= L) /* rounding guard */
                        x[3 * i + d] -= L, k += 1.0;
                    if (x[3 * i + d] < 0.0)
                        x[3 * i + d] += L, k -= 1.0;
                    if (img)
                        img[3 * i + d] += (int)k;
                }
            }
        }
        if (run_forces(n, x, type, ntypes, tab, box, fp32, F, out, nb, bonds, kb, r0)) {
            free(F);
            return -1;
        }
        double K = 0.0;
        for (int i = 0; i < n; i++) {
            double im = 1.0 / mass[i];
            for (int d = 0; d < 3; d++) {
                v[3 * i + d] += 0.5 * dt * F[3 * i + d] * im; /* B */
                K += 0.5 * mass[i] * v[3 * i + d] * v[3 * i + d];
            }
        }
        if (thermo) {
            double *t = &thermo[(long)s * 11];
            t[0] = out[0];
            t[1] = out[1];
            t[2] = K;
            for (int q = 0; q < 6; q++)
                t[3 + q] = out[2 + q];
            t[9] = out[8];
            t[10] = out[9];
        }
    }
    free(F);
    return 0;
}
