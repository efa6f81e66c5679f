/*
 * Oracle (test infrastructure only): FP64 direct Green's-function sum.
 *
 * Eq. greenSum of Appendix A:  P(x) = sum_{x'} G(x, x') f(x') h^2(x'),
 * with the free-space Green's function of Eq. green2D,
 *   G(x, x') = (1 / 2 pi) log |x - x'|.
 *
 * The paper does not say what happens when a target coincides with a source
 * (the self cell of a grid target) or comes very close to one (an off-grid
 * surface target).  This oracle takes the reading stated in the design notes:
 * the distance is clamped from below at rho_h = h * exp(c0),
 * c0 = pi/4 - 3/2 - log(2)/2, which makes the self term equal to the exact
 * mean of log r over a square cell of side h.  The caller passes rho_h.
 *
 * Plain loops in FP64, one OpenMP thread team over targets.  No blocking, no
 * expansions, no reordering of the sum beyond the loop over sources.  The
 * running sum is compensated (Neumaier's variant of Kahan summation): the
 * rounding error of each addition is carried in a second accumulator, so the
 * result does not drift by ~eps sqrt(N) as a plain sum of N terms does.
 * Built with contraction off, so no multiply-add is fused on any host.
 */
#include <math.h>
#include <stdint.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* P[t] = (1/2pi) * sum_s q[s] * log(max(|x_t - x_s|, rho_h))  for t in [0, n_tgt) */
void oracle_green_sum(int64_t n_src, const double* xs, const double* ys, const double* q,
                      int64_t n_tgt, const double* xt, const double* yt, double rho_h,
                      int nthreads, double* P)
{
    const double two_pi = 6.283185307179586476925286766559;
#ifdef _OPENMP
    /* nthreads <= 0: the OpenMP default; the choice applies to this call only */
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
    for (int64_t t = 0; t < n_tgt; ++t) {
        double acc = 0.0, err = 0.0;
        for (int64_t s = 0; s < n_src; ++s) {
            double dx = xt[t] - xs[s];
            double dy = yt[t] - ys[s];
            double r = sqrt(dx * dx + dy * dy);
            if (r < rho_h) r = rho_h;
            double term = q[s] * log(r);
            double sum = acc + term;
            /* the part of the smaller operand that the addition rounded away */
            if (fabs(acc) >= fabs(term))
                err += (acc - sum) + term;
            else
                err += (term - sum) + acc;
            acc = sum;
        }
        P[t] = (acc + err) / two_pi;
    }
}

/* The same sum over sources of different cell sizes (a multiresolution grid): source s
 * is clamped at its own rho[s] (h_s exp(c0) for a cell of side h_s, so each cell's self
 * term is its own mean of log r).
 * P[t] = (1/2pi) * sum_s q[s] * log(max(|x_t - x_s|, rho[s])), compensated as above. */
void oracle_green_sum_var(int64_t n_src, const double* xs, const double* ys, const double* q,
                          const double* rho, int64_t n_tgt, const double* xt, const double* yt,
                          int nthreads, double* P)
{
    const double two_pi = 6.283185307179586476925286766559;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
#endif
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
    for (int64_t t = 0; t < n_tgt; ++t) {
        double acc = 0.0, err = 0.0;
        for (int64_t s = 0; s < n_src; ++s) {
            double dx = xt[t] - xs[s];
            double dy = yt[t] - ys[s];
            double r = sqrt(dx * dx + dy * dy);
            if (r < rho[s]) r = rho[s];
            double term = q[s] * log(r);
            double sum = acc + term;
            if (fabs(acc) >= fabs(term))
                err += (acc - sum) + term;
            else
                err += (term - sum) + acc;
            acc = sum;
        }
        P[t] = (acc + err) / two_pi;
    }
}

/* Number of threads oracle_green_sum uses for this nthreads (1 without OpenMP). */
int oracle_max_threads(int nthreads)
{
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}
