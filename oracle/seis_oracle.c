/*
 * seis_oracle.c -- plain, slow, FP64 CPU oracle of the CMP / CRS semblance search.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and its
 * Python binding) may link, import or call this file.  It is used by the test suite,
 * by the smoke check and by the benchmark's CPU-baseline leg, and by nothing else.
 * It shares no code, header, table or helper with the CUDA implementation.
 *
 * What it computes (paper: "Massively Scaling Seismic Processing on Sunway TaihuLight
 * Supercomputer", arXiv:1907.11678):
 *
 *   - Section 2.1 / Eq. 1: for every output time sample t0 = n*dt of a gather and every
 *     candidate stacking parameter, intersect each trace with the traveltime curve,
 *     linearly interpolate the amplitude there, and form the windowed semblance
 *         S = sum_j (sum_i v_ij)^2 / (N * sum_j sum_i v_ij^2)
 *     with N the number of traces that take part (the paper prints Eq. 1 without the
 *     1/N factor; with it S lies in [0,1]).
 *   - Algorithm 1 (the per-pair loop over traces and window samples): the window runs
 *     along the trace around its own intersection k, reading samples k+j and k+j+1
 *     with one shared interpolation fraction x for all j, and accumulates num[j],
 *     den and the linear stack accumulator ac.
 *   - Section 3.2: the best candidate of each t0 is the one with the largest semblance;
 *     the stacked trace is the stack accumulator at that candidate.
 *   - Section 2.2 / Section 3.5: CRS takes the traces of every CDP whose midpoint lies
 *     within the aperture radius of the central CDP and replaces the NMO hyperbola by
 *     the (hyperbolic, A/B/C-parameterised) CRS traveltime surface.
 *
 * Readings where the paper is silent (each is also listed in the design notes):
 *   - window: hw = floor(w/2), j = -hw..hw (w odd, so exactly w samples);
 *   - a trace takes part for a (t0, candidate) only if every sample k-hw .. k+hw+1 lies
 *     inside the trace and the traveltime is real (and, for CRS, t0 + A*dm >= 0);
 *     N counts the traces that take part; S = 0 when N == 0 or the energy is 0;
 *   - argmax ties go to the lowest candidate index;
 *   - stack = ac / (N * w) at the picked candidate (0 when N == 0);
 *   - CMP traveltime t = sqrt(t0^2 + C h^2) with C = 4/v^2 and h the half-offset;
 *   - CRS traveltime t = sqrt((t0 + A dm)^2 + B dm^2 + C h^2), dm = midpoint minus the
 *     central midpoint (the 2-D hyperbolic CRS operator in A, B, C);
 *   - gradient (not in the paper): chain rule through the traveltime and the linear
 *     interpolation with k and the participation mask held fixed;
 *   - refinement (not in the paper): projected quasi-Newton (BFGS) gradient ascent in
 *     normalised coordinates with step halving, see seis_oracle_crs_refine.
 *
 * All input arrays are the same FP32 arrays the CUDA path receives; every arithmetic
 * step here is carried out in FP64.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_MAXW 255

/* ------------------------------------------------------------------------- */
/* Candidate grid, Section 3.2: "the NMO velocity array is generated according to the
 * upper and lower bounds".  Reading: nc velocities linearly spaced, bounds included,
 * converted to C = 4/v^2 (the hyperbola t^2 = t0^2 + 4 h^2 / v^2 in half-offset h). */
void seis_oracle_velocity_grid(double vmin, double vmax, int32_t nc, double* C_out)
{
    for (int32_t c = 0; c < nc; ++c) {
        double v = (nc == 1) ? vmin : vmin + (vmax - vmin) * (double)c / (double)(nc - 1);
        C_out[c] = 4.0 / (v * v);
    }
}

/* Linear grid lo..hi with n points, both ends included (CRS parameter axes). */
void seis_oracle_linear_grid(double lo, double hi, int32_t n, double* out)
{
    for (int32_t i = 0; i < n; ++i)
        out[i] = (n == 1) ? lo : lo + (hi - lo) * (double)i / (double)(n - 1);
}

/* ------------------------------------------------------------------------- */
/* Does a trace of ns samples take part when intersected at fractional sample u?
 * (Algorithm 1 reads samples k+j and k+j+1 for j = -hw..hw, k = floor(u).) */
static int window_inside(double u, int64_t ns, int hw)
{
    if (!(u == u)) return 0;                 /* NaN */
    double kf = floor(u);
    return (kf - hw >= 0.0) && (kf + hw + 1.0 <= (double)(ns - 1));
}

/* Algorithm 1 inner loop for a trace intersected at window centre k with fraction x:
 * interpolate v = (c[j+1]-c[j])*x + c[j] along the window and accumulate the semblance
 * numerator terms, the energy and the linear stack. */
static void accumulate_window(const float* f, int64_t k, double x, int hw,
                              double* num, double* den, double* ac)
{
    for (int j = -hw; j <= hw; ++j) {
        double c0 = (double)f[k + j];
        double c1 = (double)f[k + j + 1];
        double v = (c1 - c0) * x + c0;
        num[j + hw] += v;
        *den += v * v;
        *ac += v;
    }
}

/* One intersection at fractional sample u: k = floor(u), x = u - k.  Returns 1 if the
 * trace took part. */
static int intersect(const float* f, int64_t ns, double u, int hw,
                     double* num, double* den, double* ac)
{
    if (!window_inside(u, ns, hw)) return 0;
    double kf = floor(u);
    accumulate_window(f, (int64_t)kf, u - kf, hw, num, den, ac);
    return 1;
}

/* Eq. 1 with the 1/N normalisation; 0 for an empty or energy-free window. */
static double semblance_of(const double* num, int w, double den, int64_t N)
{
    if (N == 0 || !(den > 0.0)) return 0.0;
    double nu = 0.0;
    for (int j = 0; j < w; ++j) nu += num[j] * num[j];
    return nu / ((double)N * den);
}

/* Parity bookkeeping for FP32 implementations: a (row, candidate) is flagged when some
 * trace's participation would change if u moved by +-eps samples (a mask edge sitting
 * on an interpolation knot). */
static int edge_sensitive(double u, int64_t ns, int hw, double eps)
{
    return window_inside(u - eps, ns, hw) != window_inside(u + eps, ns, hw);
}

/* All moveout terms vanish (A dm = B dm^2 = C h^2 = 0): the traveltime is exactly t0 in
 * any precision, so such a trace never makes a (row, candidate) parity-sensitive. */
static int zero_moveout(double A, double B, double C, double dm, double h)
{
    return A * dm == 0.0 && B * dm * dm == 0.0 && C * h * h == 0.0;
}

/* ------------------------------------------------------------------------- */
/* Admissible results of an FP32 evaluation (reading c5).  Where a participation test of a
 * trace sits within eps of its threshold -- a mask edge within eps samples of u, or (CRS)
 * t0 + A dm or t^2 within eps of zero -- FP32 rounding may decide it either way.  Such a
 * trace is "flagged" and its admissible outcomes are listed: not taking part (where the
 * test may exclude it), or taking part with window centre k at floor(u), or at either
 * integer next to u when u lies within eps of one, with the fraction x = u - k clamped to
 * [0, 1].  Every combination of the flagged traces' outcomes, added to the sums of the
 * other traces, gives one admissible (S, stack, N); their minimum and maximum bound what a
 * correct FP32 evaluation may return.  Entries with more than ORACLE_MAXFLAG flagged
 * traces are left unresolved (NaN bounds). */
#define ORACLE_MAXFLAG 6
#define ORACLE_EDGE_EPS 1e-3   /* samples (and samples, samples^2 for p and t^2) */

/* Optional per-entry outputs of the searches (per row for seis_oracle_crs_eval).  Any
 * pointer may be NULL. */
typedef struct {
    double* S_lo;        /* admissible range of S                                   */
    double* S_hi;
    double* stack;       /* stack ac / (N w) (t0 window: s(t0) / M(t0)) at the entry */
    double* st_lo;       /* admissible range of the stack                           */
    double* st_hi;
    int32_t* N_lo;       /* admissible range of N (t0 window: M(t0))                */
    int32_t* N_hi;
} oracle_ranges;

typedef struct {
    const float* f;      /* the trace's samples                                      */
    int slot;            /* t0 window: the output-time offset j + hw of this sample  */
    int n;               /* number of outcomes (1..3)                                */
    int64_t k[3];        /* window centre, or -1: the trace does not take part       */
    double x[3];
} flagged_trace;

static void add_outcome(flagged_trace* ft, int64_t k, double x)
{
    for (int i = 0; i < ft->n; ++i)
        if (ft->k[i] == k) return;
    ft->k[ft->n] = k;
    ft->x[ft->n] = x;
    ft->n++;
}

/* The admissible outcomes of a trace of ns samples intersected at u (NaN: no real
 * traveltime); may_drop: a near-zero p or t^2 may also exclude it.  hw = 0 gives the
 * one-sample window [k, k+1] of the t0-window semblance. */
static void list_outcomes(flagged_trace* ft, const float* f, int64_t ns, double u, int hw,
                          double eps, int may_drop, int slot)
{
    ft->f = f;
    ft->slot = slot;
    ft->n = 0;
    if (may_drop || !(u == u)) add_outcome(ft, -1, 0.0);
    if (!(u == u)) return;
    double ks[2];
    int nk = 0;
    const double K0 = floor(u + 0.5);
    if (fabs(u - K0) < eps) { ks[nk++] = K0 - 1.0; ks[nk++] = K0; }
    else ks[nk++] = floor(u);
    for (int i = 0; i < nk; ++i) {
        const double kf = ks[i];
        if (kf - hw >= 0.0 && kf + hw + 1.0 <= (double)(ns - 1)) {
            double x = u - kf;
            x = x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
            add_outcome(ft, (int64_t)kf, x);
        } else {
            add_outcome(ft, -1, 0.0);
        }
    }
}

static void widen(double v, double* lo, double* hi)
{
    if (v < *lo) *lo = v;
    if (v > *hi) *hi = v;
}

/* Range over the outcome combinations of the flagged traces for the paper's window
 * (Eq. 1, Algorithm 1); (num0, den0, ac0, N0) are the sums of the other traces.  The
 * ranges start at the nominal values (S, st, N), so they always contain them. */
static void ranges_window(const double* num0, double den0, double ac0, int64_t N0, int hw,
                          const flagged_trace* ft, int nf, double S, double st, int64_t N,
                          oracle_ranges* R, int64_t at)
{
    const int w = 2 * hw + 1;
    double slo = S, shi = S, tlo = st, thi = st, nlo = (double)N, nhi = (double)N;
    if (nf > ORACLE_MAXFLAG) {
        slo = shi = tlo = thi = NAN;
    } else if (nf > 0) {
        int pick[ORACLE_MAXFLAG] = {0};
        for (;;) {
            double num[ORACLE_MAXW], den = den0, ac = ac0;
            int64_t n = N0;
            memcpy(num, num0, sizeof(double) * (size_t)w);
            for (int q = 0; q < nf; ++q) {
                const int a = pick[q];
                if (ft[q].k[a] >= 0) {
                    accumulate_window(ft[q].f, ft[q].k[a], ft[q].x[a], hw, num, &den, &ac);
                    ++n;
                }
            }
            widen(semblance_of(num, w, den, n), &slo, &shi);
            widen(n ? ac / ((double)n * w) : 0.0, &tlo, &thi);
            widen((double)n, &nlo, &nhi);
            int q = 0;
            while (q < nf && ++pick[q] == ft[q].n) { pick[q] = 0; ++q; }
            if (q == nf) break;
        }
    }
    if (R->S_lo) R->S_lo[at] = slo;
    if (R->S_hi) R->S_hi[at] = shi;
    if (R->stack) R->stack[at] = st;
    if (R->st_lo) R->st_lo[at] = tlo;
    if (R->st_hi) R->st_hi[at] = thi;
    if (R->N_lo) R->N_lo[at] = (int32_t)nlo;
    if (R->N_hi) R->N_hi[at] = (int32_t)nhi;
}

/* The same for the t0-window semblance (reading c18): per output-time offset j the sums
 * s0[j], e0[j], M0[j] of the other traces; a flagged trace adds one interpolated sample
 * to its own slot j. */
static void ranges_t0win(const double* s0, const double* e0, const int64_t* M0, int w,
                         const flagged_trace* ft, int nf, double S, double st, int64_t N,
                         oracle_ranges* R, int64_t at)
{
    const int hw = w / 2;
    double slo = S, shi = S, tlo = st, thi = st, nlo = (double)N, nhi = (double)N;
    if (nf > ORACLE_MAXFLAG) {
        slo = shi = tlo = thi = NAN;
    } else if (nf > 0) {
        int pick[ORACLE_MAXFLAG] = {0};
        for (;;) {
            double sj[ORACLE_MAXW], ej[ORACLE_MAXW];
            int64_t Mj[ORACLE_MAXW];
            memcpy(sj, s0, sizeof(double) * (size_t)w);
            memcpy(ej, e0, sizeof(double) * (size_t)w);
            memcpy(Mj, M0, sizeof(int64_t) * (size_t)w);
            for (int q = 0; q < nf; ++q) {
                const int a = pick[q];
                const int64_t k = ft[q].k[a];
                if (k < 0) continue;
                const float* f = ft[q].f;
                const double v = ((double)f[k + 1] - (double)f[k]) * ft[q].x[a] + (double)f[k];
                sj[ft[q].slot] += v;
                ej[ft[q].slot] += v * v;
                Mj[ft[q].slot] += 1;
            }
            double num = 0.0, den = 0.0;
            for (int j = 0; j < w; ++j) {
                num += sj[j] * sj[j];
                den += (double)Mj[j] * ej[j];
            }
            widen(den > 0.0 ? num / den : 0.0, &slo, &shi);
            widen(Mj[hw] ? sj[hw] / (double)Mj[hw] : 0.0, &tlo, &thi);
            widen((double)Mj[hw], &nlo, &nhi);
            int q = 0;
            while (q < nf && ++pick[q] == ft[q].n) { pick[q] = 0; ++q; }
            if (q == nf) break;
        }
    }
    if (R->S_lo) R->S_lo[at] = slo;
    if (R->S_hi) R->S_hi[at] = shi;
    if (R->stack) R->stack[at] = st;
    if (R->st_lo) R->st_lo[at] = tlo;
    if (R->st_hi) R->st_hi[at] = thi;
    if (R->N_lo) R->N_lo[at] = (int32_t)nlo;
    if (R->N_hi) R->N_hi[at] = (int32_t)nhi;
}

/* Output row r -> (owner index, local sample n) by binary search in off[0..cnt]. */
static int64_t owner_of(const int64_t* off, int64_t cnt, int64_t r)
{
    int64_t lo = 0, hi = cnt - 1;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (off[mid] <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

static void set_threads(int32_t nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/* ------------------------------------------------------------------------- */
/* CMP semblance search (Section 2.1, Eq. 1, Algorithm 1, Section 3.2).
 *
 * traces      [trace_off[ntr]] FP32 samples; trace i = traces[trace_off[i] .. trace_off[i+1])
 * h           [ntr] half-offset of each trace (m)
 * gather_off  [G+1] trace range of each CMP gather
 * out_off     [G+1] output rows of each gather: gather g has out_off[g+1]-out_off[g]
 *             output samples t0 = n*dt[g]
 * dt          [G] sampling interval of each gather (s)
 * C           [nc] candidate C = 4/v^2 values (s^2/m^2)
 * rows        global output rows to evaluate (NULL: all rows 0..out_off[G]-1)
 * Outputs are per evaluated row (index e = 0..nrows-1); any may be NULL:
 *   S[e*nc+c], Nvalid[e*nc+c], edge[e*nc+c], best_idx[e], best_S[e], second_S[e]
 *   (largest S among the other candidates), stack[e].
 * Returns 0, or -1 on invalid arguments. */
int seis_oracle_cmp(const float* traces, const int64_t* trace_off, const float* h,
                    const int64_t* gather_off, const int64_t* out_off, const float* dt,
                    int64_t G, const float* C, int32_t nc, int32_t w,
                    const int64_t* rows, int64_t nrows,
                    double* S, int32_t* Nvalid, int8_t* edge,
                    int32_t* best_idx, double* best_S, double* second_S, double* stack,
                    double knot_eps, int32_t nthreads, oracle_ranges* R)
{
    if (w < 1 || (w % 2) == 0 || w > ORACLE_MAXW || nc < 1 || G < 1) return -1;
    const int hw = w / 2;
    const int64_t total_rows = out_off[G];
    if (!rows) nrows = total_rows;
    set_threads(nthreads);

    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < nrows; ++e) {
        const int64_t r = rows ? rows[e] : e;
        const int64_t g = owner_of(out_off, G, r);
        const int64_t n = r - out_off[g];
        const double dtg = (double)dt[g];
        const double t0 = (double)n * dtg;
        double num[ORACLE_MAXW], num0[ORACLE_MAXW];
        flagged_trace ft[ORACLE_MAXFLAG];
        int32_t bi = -1; double bs = -1.0, b2 = -1.0, bst = 0.0;
        for (int32_t c = 0; c < nc; ++c) {
            const double Cc = (double)C[c];
            double den = 0.0, ac = 0.0; int64_t N = 0; int nflag = 0;
            double den0 = 0.0, ac0 = 0.0; int64_t N0 = 0;     /* unflagged traces (R) */
            memset(num, 0, sizeof(double) * (size_t)w);
            memset(num0, 0, sizeof(double) * (size_t)w);
            for (int64_t i = gather_off[g]; i < gather_off[g + 1]; ++i) {
                const double hi = (double)h[i];
                const int64_t ns_i = trace_off[i + 1] - trace_off[i];
                const float* f = traces + trace_off[i];
                const double rad = t0 * t0 + Cc * hi * hi;            /* t^2, Section 2.1 */
                if (!(rad >= 0.0)) continue;
                const double u = sqrt(rad) / dtg;                      /* traveltime in samples */
                const int flagged = (edge || R) && !zero_moveout(0.0, 0.0, Cc, 0.0, hi) &&
                                    edge_sensitive(u, ns_i, hw, knot_eps);
                N += intersect(f, ns_i, u, hw, num, &den, &ac);
                if (!R) { nflag += flagged; continue; }
                if (flagged) {
                    if (nflag < ORACLE_MAXFLAG)
                        list_outcomes(&ft[nflag], f, ns_i, u, hw, knot_eps, 0, 0);
                    ++nflag;
                } else {
                    N0 += intersect(f, ns_i, u, hw, num0, &den0, &ac0);
                }
            }
            const double s = semblance_of(num, w, den, N);
            const double st = N ? ac / ((double)N * w) : 0.0;
            if (S) S[e * nc + c] = s;
            if (Nvalid) Nvalid[e * nc + c] = (int32_t)N;
            if (edge) edge[e * nc + c] = (int8_t)(nflag > 127 ? 127 : nflag);
            if (R) ranges_window(num0, den0, ac0, N0, hw, ft, nflag, s, st, N, R, e * nc + c);
            if (s > bs) { b2 = bs; bs = s; bi = c; bst = st; }
            else if (s > b2) b2 = s;
        }
        if (best_idx) best_idx[e] = bi;
        if (best_S) best_S[e] = bs;
        if (second_S) second_S[e] = b2;
        if (stack) stack[e] = bst;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* t0-window CMP semblance (reading c18; not the paper's method, whose window runs along
 * each trace around its own intersection, Algorithm 1).  The window runs over the
 * neighbouring output times t0' = (n + j) dt, j = -hw..hw, of the same gather, each with
 * its own traveltime (Section 2.1), and every trace gives one interpolated sample there:
 *   u = sqrt(t0'^2 + C h^2) / dt, k = floor(u), x = u - k, v = f[k] + x (f[k+1] - f[k]);
 *   the trace takes part at t0' iff k >= 0 and k + 1 <= ns - 1;
 *   s(t0') = sum of v, e(t0') = sum of v^2, M(t0') = traces taking part;
 *   S(t0) = sum_j s(t0')^2 / sum_j M(t0') e(t0')   (0 if that denominator is 0),
 * where output times outside the gather's rows contribute nothing; the stack at the pick
 * is s(t0) / M(t0) (0 if M(t0) = 0).  Same outputs as seis_oracle_cmp (Nvalid = M(t0)). */
static int sample_inside(double u, int64_t ns)
{
    if (!(u == u)) return 0;
    const double kf = floor(u);
    return kf >= 0.0 && kf + 1.0 <= (double)(ns - 1);
}

int seis_oracle_cmp_t0win(const float* traces, const int64_t* trace_off, const float* h,
                          const int64_t* gather_off, const int64_t* out_off, const float* dt,
                          int64_t G, const float* C, int32_t nc, int32_t w,
                          const int64_t* rows, int64_t nrows,
                          double* S, int32_t* Nvalid, int8_t* edge,
                          int32_t* best_idx, double* best_S, double* second_S, double* stack,
                          double knot_eps, int32_t nthreads, oracle_ranges* R)
{
    if (w < 1 || (w % 2) == 0 || w > ORACLE_MAXW || nc < 1 || G < 1) return -1;
    const int hw = w / 2;
    if (!rows) nrows = out_off[G];
    set_threads(nthreads);

    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < nrows; ++e) {
        const int64_t r = rows ? rows[e] : e;
        const int64_t g = owner_of(out_off, G, r);
        const int64_t n = r - out_off[g];
        const int64_t nrow_g = out_off[g + 1] - out_off[g];
        const double dtg = (double)dt[g];
        double sb[ORACLE_MAXW], eb[ORACLE_MAXW];         /* unflagged traces per j (R) */
        int64_t Mb[ORACLE_MAXW];
        flagged_trace ft[ORACLE_MAXFLAG];
        int32_t bi = -1; double bs = -1.0, b2 = -1.0, bst = 0.0;
        for (int32_t c = 0; c < nc; ++c) {
            const double Cc = (double)C[c];
            double num = 0.0, den = 0.0, s0 = 0.0; int64_t M0 = 0; int nflag = 0;
            for (int j = -hw; j <= hw; ++j) {
                sb[j + hw] = eb[j + hw] = 0.0;
                Mb[j + hw] = 0;
                const int64_t n2 = n + j;
                if (n2 < 0 || n2 >= nrow_g) continue;
                const double t0 = (double)n2 * dtg;
                double sj = 0.0, ej = 0.0; int64_t Mj = 0;
                for (int64_t i = gather_off[g]; i < gather_off[g + 1]; ++i) {
                    const double hi = (double)h[i];
                    const int64_t ns_i = trace_off[i + 1] - trace_off[i];
                    const double u = sqrt(t0 * t0 + Cc * hi * hi) / dtg;
                    const float* f = traces + trace_off[i];
                    const int flagged = (edge || R) && !zero_moveout(0.0, 0.0, Cc, 0.0, hi) &&
                        sample_inside(u - knot_eps, ns_i) != sample_inside(u + knot_eps, ns_i);
                    if (flagged) {
                        if (R && nflag < ORACLE_MAXFLAG)
                            list_outcomes(&ft[nflag], f, ns_i, u, 0, knot_eps, 0, j + hw);
                        ++nflag;
                    }
                    if (!sample_inside(u, ns_i)) continue;
                    const int64_t k = (int64_t)floor(u);
                    const double x = u - (double)k;
                    const double v = ((double)f[k + 1] - (double)f[k]) * x + (double)f[k];
                    sj += v;
                    ej += v * v;
                    ++Mj;
                    if (!flagged) { sb[j + hw] += v; eb[j + hw] += v * v; Mb[j + hw] += 1; }
                }
                num += sj * sj;
                den += (double)Mj * ej;
                if (j == 0) { s0 = sj; M0 = Mj; }
            }
            const double sv = (den > 0.0) ? num / den : 0.0;
            const double st = M0 ? s0 / (double)M0 : 0.0;
            if (S) S[e * nc + c] = sv;
            if (Nvalid) Nvalid[e * nc + c] = (int32_t)M0;
            if (edge) edge[e * nc + c] = (int8_t)(nflag > 127 ? 127 : nflag);
            if (R) ranges_t0win(sb, eb, Mb, w, ft, nflag, sv, st, M0, R, e * nc + c);
            if (sv > bs) { b2 = bs; bs = sv; bi = c; bst = st; }
            else if (sv > b2) b2 = sv;
        }
        if (best_idx) best_idx[e] = bi;
        if (best_S) best_S[e] = bs;
        if (second_S) second_S[e] = b2;
        if (stack) stack[e] = bst;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* CRS aperture (Section 2.2, Section 3.5): for each central gather, every trace whose
 * midpoint lies within the radius apm of the central CDP's midpoint (inclusive).  The
 * central midpoint is the midpoint of the central gather's first trace.  Traces are
 * listed in increasing trace index.  nbr_off has n_central+1 entries; nbr_trace may be
 * NULL to count only.  m_c receives the central midpoints (may be NULL). */
int seis_oracle_neighbours(const float* m, const int64_t* gather_off, int64_t G,
                           const int32_t* central, int64_t n_central, double apm,
                           int64_t* nbr_off, int32_t* nbr_trace, float* m_c)
{
    const int64_t ntr = gather_off[G];
    nbr_off[0] = 0;
    for (int64_t c = 0; c < n_central; ++c) {
        const int32_t g = central[c];
        if (g < 0 || g >= G || gather_off[g + 1] <= gather_off[g]) return -1;
        const double mg = (double)m[gather_off[g]];
        if (m_c) m_c[c] = m[gather_off[g]];
        int64_t cnt = 0;
        for (int64_t i = 0; i < ntr; ++i) {
            if (fabs((double)m[i] - mg) <= apm) {
                if (nbr_trace) nbr_trace[nbr_off[c] + cnt] = (int32_t)i;
                ++cnt;
            }
        }
        nbr_off[c + 1] = nbr_off[c] + cnt;
    }
    return 0;
}

/* CRS traveltime in samples for one trace (reading c11):
 *   t^2 = (t0 + A dm)^2 + B dm^2 + C h^2; returns 0 when the trace cannot take part
 *   (t0 + A dm < 0 or t^2 < 0).  p_out, t_out receive t0 + A dm and t (s). */
static int crs_time(double t0, double A, double B, double Cc, double dm, double hh,
                    double dtg, double* u_out, double* p_out, double* t_out)
{
    const double p = t0 + A * dm;
    const double rad = p * p + B * dm * dm + Cc * hh * hh;
    if (!(p >= 0.0) || !(rad >= 0.0)) return 0;
    const double t = sqrt(rad);
    *u_out = t / dtg;
    if (p_out) *p_out = p;
    if (t_out) *t_out = t;
    return 1;
}

/* CRS semblance search over the flattened A x B x C grid, cand = (ia*nB + ib)*nC + ic.
 * Central c uses traces nbr_trace[nbr_off[c] .. nbr_off[c+1]) with dm = m[i] - m_c[c],
 * has out_off_c[c+1]-out_off_c[c] output samples at interval dt_c[c].
 * Outputs as seis_oracle_cmp (S, Nvalid, edge are [nrows][nA*nB*nC]). */
int seis_oracle_crs(const float* traces, const int64_t* trace_off, const float* h,
                    const float* m, const int64_t* nbr_off, const int32_t* nbr_trace,
                    const float* m_c, const int64_t* out_off_c, const float* dt_c,
                    int64_t n_central,
                    const float* A, int32_t nA, const float* B, int32_t nB,
                    const float* C, int32_t nC, int32_t w,
                    const int64_t* rows, int64_t nrows,
                    double* S, int32_t* Nvalid, int8_t* edge,
                    int32_t* best_idx, double* best_S, double* second_S, double* stack,
                    double knot_eps, int32_t nthreads, oracle_ranges* R)
{
    if (w < 1 || (w % 2) == 0 || w > ORACLE_MAXW || nA < 1 || nB < 1 || nC < 1 || n_central < 1)
        return -1;
    const int hw = w / 2;
    const int64_t ncand = (int64_t)nA * nB * nC;
    const int64_t total_rows = out_off_c[n_central];
    if (!rows) nrows = total_rows;
    set_threads(nthreads);

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < nrows; ++e) {
        const int64_t r = rows ? rows[e] : e;
        const int64_t c = owner_of(out_off_c, n_central, r);
        const int64_t n = r - out_off_c[c];
        const double dtg = (double)dt_c[c];
        const double t0 = (double)n * dtg;
        const double mc = (double)m_c[c];
        double num[ORACLE_MAXW], num0[ORACLE_MAXW];
        flagged_trace ft[ORACLE_MAXFLAG];
        int32_t bi = -1; double bs = -1.0, b2 = -1.0, bst = 0.0;
        for (int64_t cand = 0; cand < ncand; ++cand) {
            const int64_t ia = cand / ((int64_t)nB * nC);
            const int64_t ib = (cand / nC) % nB;
            const int64_t ic = cand % nC;
            const double Av = (double)A[ia], Bv = (double)B[ib], Cv = (double)C[ic];
            double den = 0.0, ac = 0.0; int64_t N = 0; int nflag = 0;
            double den0 = 0.0, ac0 = 0.0; int64_t N0 = 0;     /* unflagged traces (R) */
            memset(num, 0, sizeof(double) * (size_t)w);
            memset(num0, 0, sizeof(double) * (size_t)w);
            for (int64_t q = nbr_off[c]; q < nbr_off[c + 1]; ++q) {
                const int64_t i = nbr_trace[q];
                const double dm = (double)m[i] - mc;
                const int64_t ns_i = trace_off[i + 1] - trace_off[i];
                const float* f = traces + trace_off[i];
                double u, p;
                const double rad = (t0 + Av * dm) * (t0 + Av * dm) + Bv * dm * dm
                                   + Cv * (double)h[i] * (double)h[i];
                const int exact = zero_moveout(Av, Bv, Cv, dm, (double)h[i]);
                /* participation flips for a tiny change of p = t0 + A dm or of t^2
                 * (p is exact when A dm = 0, t^2 when every moveout term is 0) */
                const int drop = (edge || R) &&
                                 ((Av * dm != 0.0 && fabs(t0 + Av * dm) < knot_eps * dtg) ||
                                  (!exact && fabs(rad) < knot_eps * dtg * dtg));
                const int real = crs_time(t0, Av, Bv, Cv, dm, (double)h[i], dtg, &u, &p, NULL);
                const int flagged = drop || ((edge || R) && real && !exact &&
                                             edge_sensitive(u, ns_i, hw, knot_eps));
                if (real) N += intersect(f, ns_i, u, hw, num, &den, &ac);
                if (!R) { nflag += flagged; continue; }
                if (flagged) {
                    const double ua = real ? u : sqrt(rad > 0.0 ? rad : 0.0) / dtg;
                    if (nflag < ORACLE_MAXFLAG)
                        list_outcomes(&ft[nflag], f, ns_i, ua, hw, knot_eps, drop, 0);
                    ++nflag;
                } else if (real) {
                    N0 += intersect(f, ns_i, u, hw, num0, &den0, &ac0);
                }
            }
            const double s = semblance_of(num, w, den, N);
            const double st = N ? ac / ((double)N * w) : 0.0;
            if (S) S[e * ncand + cand] = s;
            if (Nvalid) Nvalid[e * ncand + cand] = (int32_t)N;
            if (edge) edge[e * ncand + cand] = (int8_t)(nflag > 127 ? 127 : nflag);
            if (R) ranges_window(num0, den0, ac0, N0, hw, ft, nflag, s, st, N, R,
                                 e * ncand + cand);
            if (s > bs) { b2 = bs; bs = s; bi = (int32_t)cand; bst = st; }
            else if (s > b2) b2 = s;
        }
        if (best_idx) best_idx[e] = bi;
        if (best_S) best_S[e] = bs;
        if (second_S) second_S[e] = b2;
        if (stack) stack[e] = bst;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* t0-window CRS semblance (reading c18 with the CRS traveltime of Section 2.2): as
 * seis_oracle_cmp_t0win, the window running over the central's output times t0' =
 * (n + j) dt, every aperture trace giving one interpolated sample at the traveltime
 * sqrt((t0' + A dm)^2 + B dm^2 + C h^2) when t0' + A dm >= 0, the radicand >= 0 and both
 * interpolation samples lie inside the trace.  Same outputs as seis_oracle_crs. */
int seis_oracle_crs_t0win(const float* traces, const int64_t* trace_off, const float* h,
                          const float* m, const int64_t* nbr_off, const int32_t* nbr_trace,
                          const float* m_c, const int64_t* out_off_c, const float* dt_c,
                          int64_t n_central,
                          const float* A, int32_t nA, const float* B, int32_t nB,
                          const float* C, int32_t nC, int32_t w,
                          const int64_t* rows, int64_t nrows,
                          double* S, int32_t* Nvalid, int8_t* edge,
                          int32_t* best_idx, double* best_S, double* second_S, double* stack,
                          double knot_eps, int32_t nthreads, oracle_ranges* R)
{
    if (w < 1 || (w % 2) == 0 || w > ORACLE_MAXW || nA < 1 || nB < 1 || nC < 1 || n_central < 1)
        return -1;
    const int hw = w / 2;
    const int64_t ncand = (int64_t)nA * nB * nC;
    if (!rows) nrows = out_off_c[n_central];
    set_threads(nthreads);

    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t e = 0; e < nrows; ++e) {
        const int64_t r = rows ? rows[e] : e;
        const int64_t c = owner_of(out_off_c, n_central, r);
        const int64_t n = r - out_off_c[c];
        const int64_t nrow_c = out_off_c[c + 1] - out_off_c[c];
        const double dtg = (double)dt_c[c];
        const double mc = (double)m_c[c];
        double sb[ORACLE_MAXW], eb[ORACLE_MAXW];         /* unflagged traces per j (R) */
        int64_t Mb[ORACLE_MAXW];
        flagged_trace ft[ORACLE_MAXFLAG];
        int32_t bi = -1; double bs = -1.0, b2 = -1.0, bst = 0.0;
        for (int64_t cand = 0; cand < ncand; ++cand) {
            const double Av = (double)A[cand / ((int64_t)nB * nC)];
            const double Bv = (double)B[(cand / nC) % nB];
            const double Cv = (double)C[cand % nC];
            double num = 0.0, den = 0.0, s0 = 0.0; int64_t M0 = 0; int nflag = 0;
            for (int j = -hw; j <= hw; ++j) {
                sb[j + hw] = eb[j + hw] = 0.0;
                Mb[j + hw] = 0;
                const int64_t n2 = n + j;
                if (n2 < 0 || n2 >= nrow_c) continue;
                const double t0 = (double)n2 * dtg;
                double sj = 0.0, ej = 0.0; int64_t Mj = 0;
                for (int64_t q = nbr_off[c]; q < nbr_off[c + 1]; ++q) {
                    const int64_t i = nbr_trace[q];
                    const double dm = (double)m[i] - mc;
                    const double hi = (double)h[i];
                    const int64_t ns_i = trace_off[i + 1] - trace_off[i];
                    const float* f = traces + trace_off[i];
                    const double rad = (t0 + Av * dm) * (t0 + Av * dm) + Bv * dm * dm + Cv * hi * hi;
                    const int exact = zero_moveout(Av, Bv, Cv, dm, hi);
                    const int drop = (edge || R) &&
                                     ((Av * dm != 0.0 && fabs(t0 + Av * dm) < knot_eps * dtg) ||
                                      (!exact && fabs(rad) < knot_eps * dtg * dtg));
                    double u, p;
                    const int real = crs_time(t0, Av, Bv, Cv, dm, hi, dtg, &u, &p, NULL);
                    const int flagged = drop || ((edge || R) && real && !exact &&
                        sample_inside(u - knot_eps, ns_i) != sample_inside(u + knot_eps, ns_i));
                    if (flagged) {
                        const double ua = real ? u : sqrt(rad > 0.0 ? rad : 0.0) / dtg;
                        if (R && nflag < ORACLE_MAXFLAG)
                            list_outcomes(&ft[nflag], f, ns_i, ua, 0, knot_eps, drop, j + hw);
                        ++nflag;
                    }
                    if (!real || !sample_inside(u, ns_i)) continue;
                    const int64_t k = (int64_t)floor(u);
                    const double x = u - (double)k;
                    const double v = ((double)f[k + 1] - (double)f[k]) * x + (double)f[k];
                    sj += v;
                    ej += v * v;
                    ++Mj;
                    if (!flagged) { sb[j + hw] += v; eb[j + hw] += v * v; Mb[j + hw] += 1; }
                }
                num += sj * sj;
                den += (double)Mj * ej;
                if (j == 0) { s0 = sj; M0 = Mj; }
            }
            const double sv = (den > 0.0) ? num / den : 0.0;
            const double st = M0 ? s0 / (double)M0 : 0.0;
            if (S) S[e * ncand + cand] = sv;
            if (Nvalid) Nvalid[e * ncand + cand] = (int32_t)M0;
            if (edge) edge[e * ncand + cand] = (int8_t)(nflag > 127 ? 127 : nflag);
            if (R) ranges_t0win(sb, eb, Mb, w, ft, nflag, sv, st, M0, R, e * ncand + cand);
            if (sv > bs) { b2 = bs; bs = sv; bi = (int32_t)cand; bst = st; }
            else if (sv > b2) b2 = sv;
        }
        if (best_idx) best_idx[e] = bi;
        if (best_S) best_S[e] = bs;
        if (second_S) second_S[e] = b2;
        if (stack) stack[e] = bst;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Semblance, stack and analytic gradient of one CRS operator per output row (readings
 * c8 and c15).  theta[e*3 + {0,1,2}] = (A, B, C) for evaluated row e.  CMP is the case
 * A = B = 0 with the gather's own traces as the neighbour list.
 *
 * Gradient, with k and the participation mask held fixed (derivative almost everywhere):
 *   du/dA = (t0 + A dm) dm / (t dt),  du/dB = dm^2 / (2 t dt),  du/dC = h^2 / (2 t dt)
 *   dv_j/dtheta = (f[k+j+1] - f[k+j]) du/dtheta
 *   dS/dtheta = (dNu * N den - Nu * N dden) / (N den)^2,  Nu = sum_j num_j^2. */
static void crs_eval_one(const float* traces, const int64_t* trace_off, const float* h,
                         const float* m, const int32_t* list, int64_t cnt, double mc,
                         double t0, double dtg, int hw, const double* th,
                         double* S_out, double* grad_out, double* stack_out, int32_t* N_out,
                         int8_t* knot_out, double knot_eps, oracle_ranges* R, int64_t at)
{
    int knot = 0;
    const int w = 2 * hw + 1;
    double num[ORACLE_MAXW], dnum[3][ORACLE_MAXW], num0[ORACLE_MAXW];
    double den = 0.0, ac = 0.0, dden[3] = {0.0, 0.0, 0.0};
    double den0 = 0.0, ac0 = 0.0;                 /* unflagged traces (R, reading c5) */
    int64_t N = 0, N0 = 0;
    int nflag = 0;
    flagged_trace ft[ORACLE_MAXFLAG];
    memset(num, 0, sizeof(num));
    memset(dnum, 0, sizeof(dnum));
    memset(num0, 0, sizeof(num0));
    for (int64_t q = 0; q < cnt; ++q) {
        const int64_t i = list[q];
        const double dm = (double)m[i] - mc;
        const double hh = (double)h[i];
        const int64_t ns_i = trace_off[i + 1] - trace_off[i];
        double u = 0.0, p = 0.0, t = 0.0;
        const int real = crs_time(t0, th[0], th[1], th[2], dm, hh, dtg, &u, &p, &t);
        if (R) {
            const double eps = ORACLE_EDGE_EPS;
            const double pp = t0 + th[0] * dm;
            const double rad = pp * pp + th[1] * dm * dm + th[2] * hh * hh;
            const int exact = zero_moveout(th[0], th[1], th[2], dm, hh);
            const int drop = (th[0] * dm != 0.0 && fabs(pp) < eps * dtg) ||
                             (!exact && fabs(rad) < eps * dtg * dtg);
            const int flagged = drop || (real && !exact && edge_sensitive(u, ns_i, hw, eps));
            if (flagged) {
                const double ua = real ? u : sqrt(rad > 0.0 ? rad : 0.0) / dtg;
                if (nflag < ORACLE_MAXFLAG)
                    list_outcomes(&ft[nflag], traces + trace_off[i], ns_i, ua, hw, eps, drop, 0);
                ++nflag;
            } else if (real) {
                N0 += intersect(traces + trace_off[i], ns_i, u, hw, num0, &den0, &ac0);
            }
        }
        if (!real) continue;
        /* knot bookkeeping for FP32 parity of the gradient (defined almost everywhere):
         * u within the FP32 error of u of a sample, or a mask edge within it */
        if (knot_out && !zero_moveout(th[0], th[1], th[2], dm, hh)) {
            const double tol = knot_eps * (1.0 + 3.0e-3 * u);
            if (fabs(u - floor(u + 0.5)) < tol || edge_sensitive(u, ns_i, hw, tol)) knot = 1;
        }
        if (!window_inside(u, ns_i, hw)) continue;
        const float* f = traces + trace_off[i];
        const double kf = floor(u);
        const int64_t k = (int64_t)kf;
        const double x = u - kf;
        double du[3] = {0.0, 0.0, 0.0};
        if (t > 0.0) {
            du[0] = p * dm / (t * dtg);
            du[1] = dm * dm / (2.0 * t * dtg);
            du[2] = hh * hh / (2.0 * t * dtg);
        }
        for (int j = -hw; j <= hw; ++j) {
            const double c0 = (double)f[k + j], c1 = (double)f[k + j + 1];
            const double d = c1 - c0;
            const double v = d * x + c0;
            num[j + hw] += v;
            den += v * v;
            ac += v;
            for (int a = 0; a < 3; ++a) {
                dnum[a][j + hw] += d * du[a];
                dden[a] += 2.0 * v * d * du[a];
            }
        }
        ++N;
    }
    double nu = 0.0, dnu[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < w; ++j) {
        nu += num[j] * num[j];
        for (int a = 0; a < 3; ++a) dnu[a] += 2.0 * num[j] * dnum[a][j];
    }
    if (N == 0 || !(den > 0.0)) {
        *S_out = 0.0;
        if (grad_out) grad_out[0] = grad_out[1] = grad_out[2] = 0.0;
    } else {
        const double D = (double)N * den;
        *S_out = nu / D;
        if (grad_out)
            for (int a = 0; a < 3; ++a)
                grad_out[a] = (dnu[a] * D - nu * (double)N * dden[a]) / (D * D);
    }
    if (stack_out) *stack_out = N ? ac / ((double)N * w) : 0.0;
    if (N_out) *N_out = (int32_t)N;
    if (knot_out) *knot_out = (int8_t)knot;
    if (R) {
        const double S = (N == 0 || !(den > 0.0)) ? 0.0 : nu / ((double)N * den);
        ranges_window(num0, den0, ac0, N0, hw, ft, nflag, S, N ? ac / ((double)N * w) : 0.0, N,
                      R, at);
    }
}

/* Evaluate S, dS/d(A,B,C) and the stack at given operators, one per row. */
int seis_oracle_crs_eval(const float* traces, const int64_t* trace_off, const float* h,
                         const float* m, const int64_t* nbr_off, const int32_t* nbr_trace,
                         const float* m_c, const int64_t* out_off_c, const float* dt_c,
                         int64_t n_central, int32_t w,
                         const int64_t* rows, int64_t nrows, const double* theta,
                         double* S, double* grad, double* stack, int32_t* Nvalid,
                         int8_t* knot, double knot_eps, int32_t nthreads, oracle_ranges* R)
{
    if (w < 1 || (w % 2) == 0 || w > ORACLE_MAXW || n_central < 1) return -1;
    const int hw = w / 2;
    if (!rows) nrows = out_off_c[n_central];
    set_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < nrows; ++e) {
        const int64_t r = rows ? rows[e] : e;
        const int64_t c = owner_of(out_off_c, n_central, r);
        const int64_t n = r - out_off_c[c];
        const double dtg = (double)dt_c[c];
        double s, st; int32_t N;
        crs_eval_one(traces, trace_off, h, m, nbr_trace + nbr_off[c], nbr_off[c + 1] - nbr_off[c],
                     (double)m_c[c], (double)n * dtg, dtg, hw, theta + 3 * e,
                     &s, grad ? grad + 3 * e : NULL, &st, &N, knot ? knot + e : NULL, knot_eps,
                     R, e);
        if (S) S[e] = s;
        if (stack) stack[e] = st;
        if (Nvalid) Nvalid[e] = N;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 3-vector and 3x3 helpers of the refinement. */
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double* a) { return sqrt(dot3(a, a)); }
static void mat3_vec(double H[3][3], const double* v, double* out)
{
    for (int i = 0; i < 3; ++i) out[i] = H[i][0] * v[0] + H[i][1] * v[1] + H[i][2] * v[2];
}
/* H = (step0/|g|) I: the first step along g has length step0. */
static void reset_inverse_curvature(double H[3][3], const double* g, double step0)
{
    const double gn = norm3(g);
    const double h0 = gn > 0.0 ? step0 / gn : 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] = (i == j) ? h0 : 0.0;
}
/* BFGS update of the inverse curvature estimate with step s and gradient change y (s.y > 0):
 * H <- (I - rho s y') H (I - rho y s') + rho s s', rho = 1/(s.y), written as matrix products. */
static void bfgs_inverse_update(double H[3][3], const double* s, const double* y, double sy)
{
    const double rho = 1.0 / sy;
    double L[3][3], T[3][3], N[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) L[i][j] = (i == j ? 1.0 : 0.0) - rho * s[i] * y[j];
    for (int i = 0; i < 3; ++i)                        /* T = L H */
        for (int j = 0; j < 3; ++j)
            T[i][j] = L[i][0] * H[0][j] + L[i][1] * H[1][j] + L[i][2] * H[2][j];
    for (int i = 0; i < 3; ++i)                        /* N = T L' + rho s s' */
        for (int j = 0; j < 3; ++j)
            N[i][j] = T[i][0] * L[j][0] + T[i][1] * L[j][1] + T[i][2] * L[j][2] +
                      rho * s[i] * s[j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] = N[i][j];
}

/* The BFGS update of a 3x3 inverse curvature estimate H (row-major, in place) with step s
 * and gradient change y, as the refinement applies it (exported for the pins). */
void seis_oracle_bfgs_inverse_update(double* H9, const double* s, const double* y)
{
    double H[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[i][j] = H9[3 * i + j];
    bfgs_inverse_update(H, s, y, dot3(s, y));
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H9[3 * i + j] = H[i][j];
}

/* Gradient-ascent refinement of the CRS operator from a coarse pick (reading c16).
 * Per row, in normalised coordinates z = (theta - lo) / (hi - lo), g = dS/dz, a projected
 * quasi-Newton (BFGS) ascent with step halving:
 *   evaluate S(z0), g(z0); H = (step0/|g|) I (the inverse curvature estimate); a = 1;
 *   repeat `steps` times:
 *     if |g| == 0 stop;
 *     d = H g; if d.g <= 0 reset H = (step0/|g|) I and d = H g;
 *     if |d| > 0.25 shrink d to length 0.25;
 *     trial z' = clamp(z + a d, 0, 1); evaluate S(z'), g(z');
 *     if S(z') >= S(z): with s = z' - z, y = g - g' (the gradient change of -S), and
 *       s.y > 1e-6 |s||y|, update H <- (I - s y'/s.y) H (I - y s'/s.y) + s s'/s.y;
 *       accept (z, S, g) <- (z', S', g'); a = 1;
 *     else a <- a/2.
 * Outputs theta_out [nrows*3], S_out, grad_out (dS/dtheta at the final point, may be
 * NULL), stack_out (may be NULL), and traj (may be NULL): for every row e and trial it,
 * traj[(e*steps + it)*5 + 0..4] = the trial operator (A, B, C), its S, and 1 if it was
 * accepted (0 if not); trials never made (the gradient vanished) are NaN. */
int seis_oracle_crs_refine(const float* traces, const int64_t* trace_off, const float* h,
                           const float* m, const int64_t* nbr_off, const int32_t* nbr_trace,
                           const float* m_c, const int64_t* out_off_c, const float* dt_c,
                           int64_t n_central, int32_t w,
                           const int64_t* rows, int64_t nrows, const double* theta_in,
                           const double* lo3, const double* hi3, int32_t steps, double step0,
                           double* theta_out, double* S_out, double* grad_out, double* stack_out,
                           int32_t nthreads, double* traj)
{
    if (w < 1 || (w % 2) == 0 || w > ORACLE_MAXW || n_central < 1 || steps < 0) return -1;
    for (int a = 0; a < 3; ++a) if (!(hi3[a] > lo3[a])) return -1;
    const int hw = w / 2;
    if (!rows) nrows = out_off_c[n_central];
    set_threads(nthreads);
    #pragma omp parallel for schedule(dynamic, 4)
    for (int64_t e = 0; e < nrows; ++e) {
        const int64_t r = rows ? rows[e] : e;
        const int64_t c = owner_of(out_off_c, n_central, r);
        const int64_t n = r - out_off_c[c];
        const double dtg = (double)dt_c[c];
        const int32_t* list = nbr_trace + nbr_off[c];
        const int64_t cnt = nbr_off[c + 1] - nbr_off[c];
        const double t0 = (double)n * dtg, mc = (double)m_c[c];
        double z[3], th[3], g[3], gz[3], s, st;
        for (int a = 0; a < 3; ++a) {
            z[a] = (theta_in[3 * e + a] - lo3[a]) / (hi3[a] - lo3[a]);
            th[a] = theta_in[3 * e + a];
        }
        crs_eval_one(traces, trace_off, h, m, list, cnt, mc, t0, dtg, hw, th, &s, g, &st, NULL,
                     NULL, 0.0, NULL, 0);
        double span[3], H[3][3], al = 1.0;
        for (int a = 0; a < 3; ++a) span[a] = hi3[a] - lo3[a];
        for (int a = 0; a < 3; ++a) gz[a] = g[a] * span[a];
        reset_inverse_curvature(H, gz, step0);
        if (traj)
            for (int q = 0; q < 5 * steps; ++q) traj[e * 5 * steps + q] = NAN;
        for (int it = 0; it < steps; ++it) {
            for (int a = 0; a < 3; ++a) gz[a] = g[a] * span[a];
            if (!(norm3(gz) > 0.0)) break;
            double d[3];
            mat3_vec(H, gz, d);
            if (!(dot3(d, gz) > 0.0)) {
                reset_inverse_curvature(H, gz, step0);
                mat3_vec(H, gz, d);
            }
            const double dn = norm3(d);
            if (dn > 0.25) for (int a = 0; a < 3; ++a) d[a] *= 0.25 / dn;
            double z2[3], th2[3], g2[3], s2, st2;
            for (int a = 0; a < 3; ++a) {
                double zz = z[a] + al * d[a];
                z2[a] = zz < 0.0 ? 0.0 : (zz > 1.0 ? 1.0 : zz);
                th2[a] = lo3[a] + z2[a] * span[a];
            }
            crs_eval_one(traces, trace_off, h, m, list, cnt, mc, t0, dtg, hw, th2, &s2, g2, &st2,
                         NULL, NULL, 0.0, NULL, 0);
            if (traj) {
                double* tr = traj + (e * steps + it) * 5;
                tr[0] = th2[0]; tr[1] = th2[1]; tr[2] = th2[2]; tr[3] = s2;
                tr[4] = s2 >= s ? 1.0 : 0.0;
            }
            if (s2 >= s) {
                double sv[3], yv[3];
                for (int a = 0; a < 3; ++a) {
                    sv[a] = z2[a] - z[a];
                    yv[a] = g[a] * span[a] - g2[a] * span[a];
                }
                const double sy = dot3(sv, yv);
                if (sy > 1e-6 * norm3(sv) * norm3(yv)) bfgs_inverse_update(H, sv, yv, sy);
                for (int a = 0; a < 3; ++a) { z[a] = z2[a]; th[a] = th2[a]; g[a] = g2[a]; }
                s = s2; st = st2;
                al = 1.0;
            } else {
                al *= 0.5;
            }
        }
        for (int a = 0; a < 3; ++a) theta_out[3 * e + a] = th[a];
        if (S_out) S_out[e] = s;
        if (grad_out) for (int a = 0; a < 3; ++a) grad_out[3 * e + a] = g[a];
        if (stack_out) stack_out[e] = st;
    }
    return 0;
}

int seis_oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
