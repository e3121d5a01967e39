/*
 * FP64 CPU oracle for the k-superstep multidimensional complex FFT.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file; only the tests, the package's smoke check and the bench's
 * CPU-baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library.
 *
 * What it computes (paper, Section 1 and Section 2.2): the k-dimensional DFT
 *
 *   X[k_0..k_{r-1}] = sum_j x[j_0..j_{r-1}] * exp(s * 2*pi*i * sum_d j_d k_d / n_d)
 *
 * with s = -1 for the forward transform and s = +1 for the inverse, computed
 * as the paper does it: one superstep per axis, each superstep a batch of 1D
 * Cooley-Tukey FFTs along that axis (Section 1, "supersteps"; Section 4.1,
 * "Pencil Computation").  The per-pencil FFT here is the textbook iterative
 * radix-2 algorithm with an explicit bit-reversal permutation -- a different
 * ordering from both the paper's even/odd reshape and the GPU kernels, on
 * purpose.  Roots of unity are computed directly for every (m, n) in double
 * precision with quadrant/octant reduction, never by recurrence.
 *
 * Normalisation (Section 4.2, inverse transform): mode 0 scales each axis by
 * 1/n_d on the inverse only (total 1/N, numpy's ifftn); mode 1 never scales;
 * mode 2 scales each axis by 1/sqrt(n_d) in both directions.
 *
 * Layout: row-major, last axis contiguous (Section 1: input(i,j,k) is element
 * k of the pencil held by PE(i,j)); complex numbers interleaved (re, im) in
 * doubles; an outermost batch dimension of independent transforms.
 *
 * Also here: the brute-force O(N^2) DFT straight from the definition (for
 * pinning the FFT on tiny inputs) and the direct evaluation of one output
 * coefficient (for sampled checks at sizes where a full transform is too
 * slow).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846264338327950288

/* exp(s * 2*pi*i * m / n) for integer m, n > 0, s = +-1.
 * Reduction: m mod n -> quadrant q = floor(4m/n) and remainder rho in [0, n),
 * so the angle is (pi/2)(q + rho/n).  The in-quadrant angle is evaluated on
 * whichever of rho, n - rho keeps it in the first octant. */
static void unit_root(int64_t m, int64_t n, int s, double *re, double *im) {
    m %= n;
    if (m < 0) m += n;
    int64_t q = (4 * m) / n;
    int64_t rho = 4 * m - q * n;              /* in [0, n) */
    double c0, s0;
    if (2 * rho <= n) {
        double a = (OR_PI / 2.0) * (double)rho / (double)n;
        c0 = cos(a);
        s0 = sin(a);
    } else {
        double a = (OR_PI / 2.0) * (double)(n - rho) / (double)n;
        c0 = sin(a);
        s0 = cos(a);
    }
    double c, sn;
    switch (q) {
    case 0: c = c0; sn = s0; break;
    case 1: c = -s0; sn = c0; break;
    case 2: c = -c0; sn = -s0; break;
    default: c = s0; sn = -c0; break;
    }
    *re = c;
    *im = (s < 0) ? -sn : sn;
}

static int is_pow2(int64_t n) { return n > 0 && (n & (n - 1)) == 0; }

static int ilog2(int64_t n) {
    int l = 0;
    while ((int64_t)1 << l < n) ++l;
    return l;
}

/* In-place radix-2 decimation-in-time FFT of one pencil p[0..n) (interleaved).
 * w holds exp(s*2*pi*i*j/n) for j in [0, n/2).  Bit-reversal first, then
 * log2(n) levels of butterflies of span 2, 4, ..., n. */
static void fft_pencil(double *p, int64_t n, const double *w) {
    int lg = ilog2(n);
    for (int64_t i = 0; i < n; ++i) {
        int64_t r = 0;
        for (int b = 0; b < lg; ++b)
            if (i & ((int64_t)1 << b)) r |= (int64_t)1 << (lg - 1 - b);
        if (r > i) {
            double tr = p[2 * i], ti = p[2 * i + 1];
            p[2 * i] = p[2 * r];
            p[2 * i + 1] = p[2 * r + 1];
            p[2 * r] = tr;
            p[2 * r + 1] = ti;
        }
    }
    for (int64_t span = 2; span <= n; span <<= 1) {
        int64_t half = span >> 1;
        int64_t wstep = n / span;             /* root index stride for this span */
        for (int64_t base = 0; base < n; base += span) {
            for (int64_t j = 0; j < half; ++j) {
                double wr = w[2 * (j * wstep)], wi = w[2 * (j * wstep) + 1];
                double *a = p + 2 * (base + j);
                double *b = p + 2 * (base + j + half);
                double br = b[0] * wr - b[1] * wi;
                double bi = b[0] * wi + b[1] * wr;
                b[0] = a[0] - br;
                b[1] = a[1] - bi;
                a[0] = a[0] + br;
                a[1] = a[1] + bi;
            }
        }
    }
}

/* One superstep: 1D FFTs of length n along an axis viewed as
 * [outer][n][inner] (elements), each result scaled by `scale`. */
static void superstep(double *x, int64_t outer, int64_t n, int64_t inner,
                      int s, double scale) {
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)(n / 2 + 1));
    for (int64_t j = 0; j < n / 2; ++j) unit_root(j, n, s, &w[2 * j], &w[2 * j + 1]);
    int64_t npen = outer * inner;
#pragma omp parallel
    {
        double *p = (double *)malloc(sizeof(double) * 2 * (size_t)n);
#pragma omp for schedule(static)
        for (int64_t pen = 0; pen < npen; ++pen) {
            int64_t o = pen / inner, i = pen % inner;
            double *base = x + 2 * (o * n * inner + i);
            for (int64_t k = 0; k < n; ++k) {
                p[2 * k] = base[2 * k * inner];
                p[2 * k + 1] = base[2 * k * inner + 1];
            }
            if (n > 1) fft_pencil(p, n, w);
            for (int64_t k = 0; k < n; ++k) {
                base[2 * k * inner] = p[2 * k] * scale;
                base[2 * k * inner + 1] = p[2 * k + 1] * scale;
            }
        }
        free(p);
    }
    free(w);
}

static double axis_scale(int64_t n, int s, int norm) {
    if (norm == 0) return s > 0 ? 1.0 / (double)n : 1.0;
    if (norm == 2) return 1.0 / sqrt((double)n);
    return 1.0;
}

/* Return codes: 0 ok, -1 bad argument, -2 non-power-of-two size. */
static int check_dims(const int64_t *dims, int rank, int64_t batch) {
    if (rank < 1 || rank > 8 || batch < 0 || !dims) return -1;
    for (int d = 0; d < rank; ++d)
        if (!is_pow2(dims[d])) return -2;
    return 0;
}

/* Full k-dimensional transform, out-of-place (in may equal out).
 * Supersteps run from the last (contiguous) axis to the first, as the paper
 * does for its first superstep (Section 4.2); any order gives the same result
 * in exact arithmetic (Section 1). */
int oracle_fftn(const double *in, double *out, const int64_t *dims, int rank,
                int64_t batch, int sign, int norm) {
    int rc = check_dims(dims, rank, batch);
    if (rc) return rc;
    if (sign != 1 && sign != -1) return -1;
    int64_t N = 1;
    for (int d = 0; d < rank; ++d) N *= dims[d];
    if (in != out) memmove(out, in, sizeof(double) * 2 * (size_t)(N * batch));
    for (int d = rank - 1; d >= 0; --d) {
        int64_t inner = 1, outer = batch;
        for (int e = d + 1; e < rank; ++e) inner *= dims[e];
        for (int e = 0; e < d; ++e) outer *= dims[e];
        superstep(out, outer, dims[d], inner, sign, axis_scale(dims[d], sign, norm));
    }
    return 0;
}

/* One superstep alone, along `axis`, scaled by `scale`, in place. */
int oracle_fft_axis(double *x, const int64_t *dims, int rank, int64_t batch,
                    int axis, int sign, double scale) {
    int rc = check_dims(dims, rank, batch);
    if (rc) return rc;
    if (axis < 0 || axis >= rank || (sign != 1 && sign != -1)) return -1;
    int64_t inner = 1, outer = batch;
    for (int e = axis + 1; e < rank; ++e) inner *= dims[e];
    for (int e = 0; e < axis; ++e) outer *= dims[e];
    superstep(x, outer, dims[axis], inner, sign, scale);
    return 0;
}

/* Phase index of exp(s*2*pi*i*sum_d j_d k_d/n_d) written as exp(s*2*pi*i*m/N)
 * with N = prod n_d: m = sum_d (j_d k_d mod n_d) * (N / n_d) mod N. */
static int64_t phase_index(const int64_t *j, const int64_t *k, const int64_t *dims,
                           int rank, int64_t N) {
    int64_t m = 0;
    for (int d = 0; d < rank; ++d) {
        int64_t t = (j[d] * k[d]) % dims[d];
        m = (m + t * (N / dims[d])) % N;
    }
    return m;
}

static void unravel(int64_t idx, const int64_t *dims, int rank, int64_t *out) {
    for (int d = rank - 1; d >= 0; --d) {
        out[d] = idx % dims[d];
        idx /= dims[d];
    }
}

/* Brute-force O(N^2) DFT of each batch item straight from the definition,
 * with compensated (Neumaier) summation.  Unnormalised. */
int oracle_dft_brute(const double *in, double *out, const int64_t *dims, int rank,
                     int64_t batch, int sign) {
    int rc = check_dims(dims, rank, batch);
    if (rc) return rc;
    if (rank > 8 || (sign != 1 && sign != -1)) return -1;
    int64_t N = 1;
    for (int d = 0; d < rank; ++d) N *= dims[d];
    double *w = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    for (int64_t m = 0; m < N; ++m) unit_root(m, N, sign, &w[2 * m], &w[2 * m + 1]);
    for (int64_t b = 0; b < batch; ++b) {
        const double *xb = in + 2 * b * N;
        double *yb = out + 2 * b * N;
#pragma omp parallel for schedule(static)
        for (int64_t kf = 0; kf < N; ++kf) {
            int64_t k[8], j[8];
            unravel(kf, dims, rank, k);
            double sr = 0, cr = 0, si = 0, ci = 0;
            for (int64_t jf = 0; jf < N; ++jf) {
                unravel(jf, dims, rank, j);
                int64_t m = phase_index(j, k, dims, rank, N);
                double tr = xb[2 * jf] * w[2 * m] - xb[2 * jf + 1] * w[2 * m + 1];
                double ti = xb[2 * jf] * w[2 * m + 1] + xb[2 * jf + 1] * w[2 * m];
                double t = sr + tr;
                cr += (fabs(sr) >= fabs(tr)) ? (sr - t) + tr : (tr - t) + sr;
                sr = t;
                t = si + ti;
                ci += (fabs(si) >= fabs(ti)) ? (si - t) + ti : (ti - t) + si;
                si = t;
            }
            yb[2 * kf] = sr + cr;
            yb[2 * kf + 1] = si + ci;
        }
    }
    free(w);
    return 0;
}

/* Direct evaluation of selected output coefficients of one transform of
 * size prod(dims) (no batch): out[2q..2q+1] = X[kflat[q]], unnormalised.
 * O(N) per coefficient; the roots come from unit_root per term. */
int oracle_dft_points(const double *in, const int64_t *dims, int rank, int sign,
                      const int64_t *kflat, int64_t nk, double *out) {
    int rc = check_dims(dims, rank, 1);
    if (rc) return rc;
    if (rank > 8 || (sign != 1 && sign != -1)) return -1;
    int64_t N = 1;
    for (int d = 0; d < rank; ++d) N *= dims[d];
    for (int64_t q = 0; q < nk; ++q) {
        int64_t k[8];
        unravel(kflat[q], dims, rank, k);
        double sr = 0, si = 0;
#pragma omp parallel for reduction(+ : sr, si) schedule(static)
        for (int64_t jf = 0; jf < N; ++jf) {
            int64_t j[8];
            unravel(jf, dims, rank, j);
            int64_t m = phase_index(j, k, dims, rank, N);
            double wr, wi;
            unit_root(m, N, sign, &wr, &wi);
            sr += in[2 * jf] * wr - in[2 * jf + 1] * wi;
            si += in[2 * jf] * wi + in[2 * jf + 1] * wr;
        }
        out[2 * q] = sr;
        out[2 * q + 1] = si;
    }
    return 0;
}

/* exp(s*2*pi*i*m/n) exported for the pins of the root evaluation itself. */
void oracle_unit_root(int64_t m, int64_t n, int sign, double *re_im) {
    unit_root(m, n, sign, &re_im[0], &re_im[1]);
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
