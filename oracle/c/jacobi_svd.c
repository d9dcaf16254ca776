/*
 * Oracle (test infrastructure only): one-sided Jacobi SVD, Hestenes' method.
 *
 * The SVD step of Basic SSA (section 2.2) asks for the singular triples of
 * the trajectory matrix X.  This file computes them the plain way, on an
 * explicitly formed matrix, so that it can serve as the reference the fast
 * method is checked against.  Nothing here is used by the CUDA path.
 *
 * Method (Hestenes 1958; rotation formula as in Demmel & Veselic 1992):
 *   A is m x n (column-major, m >= n).  Repeat cyclic sweeps over all column
 *   pairs (p, q), p < q.  For each pair with
 *       alpha = a_p.a_p, beta = a_q.a_q, gamma = a_p.a_q,
 *   and |gamma| > tol * sqrt(alpha * beta), apply the plane rotation
 *       zeta = (beta - alpha) / (2 gamma),
 *       t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),  c = 1/sqrt(1+t^2), s = c t,
 *       a_p <- c a_p - s a_q,   a_q <- s a_p + c a_q,
 *   and the same rotation to columns p, q of W (initially the identity).
 *   Stop after a sweep with no rotation.  Then A = (A W^T) ... i.e. the
 *   original matrix equals Anew W^T, the columns of Anew are mutually
 *   orthogonal, sigma_i = ||Anew_i||, and the right singular vectors are
 *   the columns of W.
 * Returns the number of sweeps used, or -1 if max_sweeps was reached.
 */
#include <math.h>
#include <stddef.h>

int oracle_jacobi_svd(int m, int n, double *A, double *W, double tol, int max_sweeps)
{
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i)
            W[(size_t)j * n + i] = (i == j) ? 1.0 : 0.0;
    for (int sweep = 1; sweep <= max_sweeps; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < n - 1; ++p) {
            for (int q = p + 1; q < n; ++q) {
                double *ap = A + (size_t)p * m, *aq = A + (size_t)q * m;
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int i = 0; i < m; ++i) {
                    alpha += ap[i] * ap[i];
                    beta += aq[i] * aq[i];
                    gamma += ap[i] * aq[i];
                }
                if (alpha == 0.0 || beta == 0.0) continue;
                if (fabs(gamma) <= tol * sqrt(alpha) * sqrt(beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int i = 0; i < m; ++i) {
                    double x = ap[i], y = aq[i];
                    ap[i] = c * x - s * y;
                    aq[i] = s * x + c * y;
                }
                double *wp = W + (size_t)p * n, *wq = W + (size_t)q * n;
                for (int i = 0; i < n; ++i) {
                    double x = wp[i], y = wq[i];
                    wp[i] = c * x - s * y;
                    wq[i] = s * x + c * y;
                }
            }
        }
        if (!rotated) return sweep;
    }
    return -1;
}
