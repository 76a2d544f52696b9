/*
 * Seeded-input generator: exact line/pixel intersection lengths (Siddon's
 * method) for a 2-D parallel-beam scan of an n x n image, written as CSR.
 *
 * This is input generation, not part of the reconstruction method: the paper
 * takes the X-ray projection model A as given (Sec. 1, Eq. 1).  Both the CPU
 * oracle and the GPU library consume the CSR produced here.
 *
 * Geometry (fixed convention, identical on every machine):
 *   pixel (s,t) covers x in [t - n/2, t + 1 - n/2), y in [n/2 - s - 1, n/2 - s)
 *   ray (k,d) is the line  x cos(th_k) + y sin(th_k) = u_d,
 *     th_k = k * pi / n_angles,  u_d = d - (n_bins - 1)/2   (unit bins)
 *   row index = k * n_bins + d, column index = s * n + t.
 * The weight of (ray, pixel) is the exact length of the chord inside the
 * pixel.  The ray is cut at every grid line it crosses; each piece goes to the
 * pixel holding its midpoint (half-open pixels, so a ray running exactly along
 * a grid line is given to the pixel on the + side of that line).  sin/cos
 * smaller than 1e-15 in magnitude are taken as 0, pieces of length <= 1e-12
 * are dropped, and columns are ascending within a row.
 *
 * Build with -ffp-contract=off so that x86 and aarch64 give identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define SNAP_EPS 1e-15
#define SEG_EPS 1e-12

typedef struct {
    int32_t col;
    double w;
} entry_t;

/* Walks one ray; writes at most 2n+2 entries into out (sorted by column).
 * Returns the number of entries. */
static int trace_ray(int n, double th, double u, entry_t *out, double *alpha_buf) {
    double c = cos(th), s = sin(th);
    if (fabs(c) < SNAP_EPS) c = 0.0;
    if (fabs(s) < SNAP_EPS) s = 0.0;
    const double h = 0.5 * (double)n;
    /* P(a) = (u c - a s, u s + a c), unit speed. */
    const double x0 = u * c, y0 = u * s;
    double amin = -INFINITY, amax = INFINITY;
    if (s != 0.0) {
        double a1 = (x0 - h) / s, a2 = (x0 + h) / s;
        if (a1 > a2) { double tmp = a1; a1 = a2; a2 = tmp; }
        if (a1 > amin) amin = a1;
        if (a2 < amax) amax = a2;
    } else if (fabs(x0) > h) {
        return 0;
    }
    if (c != 0.0) {
        double a1 = (-h - y0) / c, a2 = (h - y0) / c;
        if (a1 > a2) { double tmp = a1; a1 = a2; a2 = tmp; }
        if (a1 > amin) amin = a1;
        if (a2 < amax) amax = a2;
    } else if (fabs(y0) > h) {
        return 0;
    }
    if (!(amax - amin > SEG_EPS)) return 0;

    /* Crossings with vertical lines x = -h + k and horizontal lines y = -h + l,
     * each list generated in increasing alpha, then merged. */
    int nv = 0, nh = 0;
    double *av = alpha_buf, *ah = alpha_buf + (n + 1);
    if (s != 0.0) {
        for (int k = 0; k <= n; ++k) {
            int kk = (s > 0.0) ? (n - k) : k; /* alpha = (x0 - X)/s decreasing in X when s > 0 */
            double X = -h + (double)kk;
            double a = (x0 - X) / s;
            if (a > amin && a < amax) av[nv++] = a;
        }
    }
    if (c != 0.0) {
        for (int l = 0; l <= n; ++l) {
            int ll = (c > 0.0) ? l : (n - l); /* alpha = (Y - y0)/c increasing in Y when c > 0 */
            double Y = -h + (double)ll;
            double a = (Y - y0) / c;
            if (a > amin && a < amax) ah[nh++] = a;
        }
    }
    int cnt = 0;
    double prev = amin;
    int iv = 0, ih = 0;
    int last_col = -1;
    for (;;) {
        double next;
        if (iv < nv && (ih >= nh || av[iv] <= ah[ih])) next = av[iv++];
        else if (ih < nh) next = ah[ih++];
        else next = amax;
        double len = next - prev;
        if (len > SEG_EPS) {
            double mid = 0.5 * (prev + next);
            double xm = x0 - mid * s, ym = y0 + mid * c;
            double ft = floor(xm + h), fy = floor(ym + h);
            if (ft >= 0.0 && ft < (double)n && fy >= 0.0 && fy < (double)n) {
                int t = (int)ft, srow = n - 1 - (int)fy;
                int col = srow * n + t;
                if (col == last_col) {
                    out[cnt - 1].w += len;
                } else {
                    out[cnt].col = col;
                    out[cnt].w = len;
                    ++cnt;
                    last_col = col;
                }
            }
        }
        prev = next;
        if (next == amax) break;
    }
    /* Order by column.  Along the ray the row s is monotone and, inside one
     * image row, t is monotone, so reversing runs is enough. */
    if (cnt > 1 && out[0].col > out[cnt - 1].col) {
        for (int i = 0, j = cnt - 1; i < j; ++i, --j) { entry_t tmp = out[i]; out[i] = out[j]; out[j] = tmp; }
    }
    int i = 0;
    while (i < cnt) {
        int row = out[i].col / n;
        int j = i;
        while (j + 1 < cnt && out[j + 1].col / n == row) ++j;
        if (j > i && out[i].col > out[j].col) {
            for (int a = i, b = j; a < b; ++a, --b) { entry_t tmp = out[a]; out[a] = out[b]; out[b] = tmp; }
        }
        i = j + 1;
    }
    return cnt;
}

/* Pass 1: number of nonzeros of every row.  row_nnz has n_angles*n_bins entries. */
void siddon_count(int n, int n_angles, int n_bins, int64_t *row_nnz) {
    const double pi = 3.14159265358979323846;
#pragma omp parallel
    {
        entry_t *buf = (entry_t *)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
        double *abuf = (double *)malloc(sizeof(double) * (size_t)(2 * n + 4));
#pragma omp for schedule(static)
        for (int k = 0; k < n_angles; ++k) {
            double th = (double)k * pi / (double)n_angles;
            for (int d = 0; d < n_bins; ++d) {
                double u = (double)d - 0.5 * (double)(n_bins - 1);
                row_nnz[(int64_t)k * n_bins + d] = trace_ray(n, th, u, buf, abuf);
            }
        }
        free(buf);
        free(abuf);
    }
}

/* Pass 2: fill columns and weights at the offsets given by row_ptr. */
void siddon_fill(int n, int n_angles, int n_bins, const int64_t *row_ptr, int32_t *cols, double *vals) {
    const double pi = 3.14159265358979323846;
#pragma omp parallel
    {
        entry_t *buf = (entry_t *)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
        double *abuf = (double *)malloc(sizeof(double) * (size_t)(2 * n + 4));
#pragma omp for schedule(static)
        for (int k = 0; k < n_angles; ++k) {
            double th = (double)k * pi / (double)n_angles;
            for (int d = 0; d < n_bins; ++d) {
                double u = (double)d - 0.5 * (double)(n_bins - 1);
                int64_t row = (int64_t)k * n_bins + d;
                int cnt = trace_ray(n, th, u, buf, abuf);
                int64_t o = row_ptr[row];
                for (int e = 0; e < cnt; ++e) {
                    cols[o + e] = buf[e].col;
                    vals[o + e] = buf[e].w;
                }
            }
        }
        free(buf);
        free(abuf);
    }
}

/* Single ray, for tests: returns the entry count, fills cols/vals (capacity 2n+2). */
int siddon_ray(int n, double theta, double u, int32_t *cols, double *vals) {
    entry_t *buf = (entry_t *)malloc(sizeof(entry_t) * (size_t)(2 * n + 4));
    double *abuf = (double *)malloc(sizeof(double) * (size_t)(2 * n + 4));
    int cnt = trace_ray(n, theta, u, buf, abuf);
    for (int e = 0; e < cnt; ++e) {
        cols[e] = buf[e].col;
        vals[e] = buf[e].w;
    }
    free(buf);
    free(abuf);
    return cnt;
}
