/* Oracle: the pair sum of the discrete photoionization model in plain C.
 *
 * TEST INFRASTRUCTURE ONLY: part of the CPU oracle (tests, smoke check and the
 * CPU baseline of the benchmark); the product path never links it.
 *
 * Sec. 3, Eq. (summation): out_i = sum_{j != i} K(|x_i - y_j|) q_j with the
 * kernel of Eq. (gfun), K(R) = (e^{-aR} - e^{-bR}) / (4 pi R^3 ln(b/a)),
 * written as -e^{-aR} expm1(-(b-a)R) / (4 pi R^3 ln(b/a)). FP64 throughout,
 * targets split over OpenMP threads, sources summed in input order.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_direct_sum(int64_t nt, const double* tgt, const int64_t* tidx,
                       int64_t ns, const double* src, const int64_t* sidx, const double* q,
                       double a, double b, double* out) {
    const double norm = 1.0 / (4.0 * M_PI * log(b / a));
    const double bma = b - a;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < nt; ++i) {
        const double x = tgt[3 * i], y = tgt[3 * i + 1], z = tgt[3 * i + 2];
        double s = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            if (sidx[j] == tidx[i]) continue;
            const double dx = x - src[3 * j], dy = y - src[3 * j + 1], dz = z - src[3 * j + 2];
            const double R = sqrt(dx * dx + dy * dy + dz * dz);
            const double k = -exp(-a * R) * expm1(-bma * R) * norm / (R * R * R);
            s += k * q[j];
        }
        out[i] = s;
    }
}
