/*
 * FP64 CPU oracle of the DiffCloud mesh-to-point-cloud loss and its vertex gradient.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously-correct statement of what
 * the CUDA path computes. Only the tests, the smoke check and the bench's CPU-baseline leg
 * load it; the library never does. It shares no code, header or table with the CUDA path.
 *
 * What it computes, per frame (paper Section III):
 *   - face areas A_f = 1/2 |(p2 - p1) x (p3 - p1)| and their inclusive prefix sum C_f,
 *     A = C_{F-1}                                            (Sec. III-B, area weighting)
 *   - face pick f_i = min{ f : C_f > r_f,i * A }              (Sec. III-B, area weighting)
 *   - barycentric point x_i = w0 p_f0 + w1 p_f1 + w2 p_f2 with
 *     w = (1 - sqrt(r1), sqrt(r1) (1 - r2), sqrt(r1) r2)       (Eq. 3)
 *   - brute-force nearest neighbours in both directions       (Eq. 1 / Eq. 2)
 *   - L_t = mean_i min_j |x_i - y_j|^2 + mean_j min_i |y_j - x_i|^2   (Eq. 1)
 *     or  L_t = sum_i min_j |x_i - y_j|^2                      (Eq. 2)
 *   - dL/dx_i along the chosen neighbour, scattered to the face's vertices with the
 *     barycentric weights as the partial derivatives           (Eq. 4)
 *
 * Precision. Areas, prefix sums, face picks, points, losses and gradients are in double,
 * from the float32 inputs promoted exactly. The one decision that floating point turns into
 * an integer on the CUDA path as well -- which neighbour is nearest -- is taken here in
 * float32 with a stated evaluation order (x32, d32 below), so both sides decide in the same
 * precision; every quantity that is reported as a value uses double.
 *
 *   float32 point:    s = sqrt(r1); w0 = 1 - s; w1 = s * (1 - r2); w2 = s * r2;
 *                     x = fma(w2, p2, fma(w1, p1, w0 * p0))      per coordinate
 *   float32 distance: dx = a - b (per coordinate);  d = fma(dz, dz, fma(dy, dy, dx * dx))
 *   ties:             the lowest index among equal minima wins.
 *
 * Compile with -ffp-contract=off so the compiler adds no fused operations of its own.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_EDEGENERATE (-2)

#define ORC_BIDIR_MEAN 0 /* Eq. 1 */
#define ORC_UNIDIR_SUM 1 /* Eq. 2 */

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel neighbour search (for timing on one core or all of them). */
void orc_set_num_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* Sec. III-B: area of every face, 1/2 |(p2 - p1) x (p3 - p1)|, in double. */
void orc_face_areas(const float* verts, const int32_t* faces, int F, double* area) {
    for (int f = 0; f < F; ++f) {
        const float* p1 = verts + 3 * (int64_t)faces[3 * f + 0];
        const float* p2 = verts + 3 * (int64_t)faces[3 * f + 1];
        const float* p3 = verts + 3 * (int64_t)faces[3 * f + 2];
        double e1[3], e2[3], c[3];
        for (int k = 0; k < 3; ++k) {
            e1[k] = (double)p2[k] - (double)p1[k];
            e2[k] = (double)p3[k] - (double)p1[k];
        }
        c[0] = e1[1] * e2[2] - e1[2] * e2[1];
        c[1] = e1[2] * e2[0] - e1[0] * e2[2];
        c[2] = e1[0] * e2[1] - e1[1] * e2[0];
        area[f] = 0.5 * sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    }
}

/* Sec. IV-F (fold scenario) and Sec. IV-C (the regressors' training clouds): points are
 * sampled from a subset of the faces only. A face outside the subset (mask[f] == 0) gets
 * area weight 0, so the inverse-CDF pick below never selects it. */
void orc_mask_areas(double* area, const uint8_t* mask, int F) {
    for (int f = 0; f < F; ++f)
        if (!mask[f]) area[f] = 0.0;
}

/* Sec. III-B: inclusive prefix sum of the areas, summed in face order. */
void orc_area_cdf(const double* area, int F, double* cdf) {
    double acc = 0.0;
    for (int f = 0; f < F; ++f) {
        acc += area[f];
        cdf[f] = acc;
    }
}

/* Sec. III-B: pick a face with probability proportional to its area by inverting the CDF:
 * the first f whose cumulative area exceeds r * A (strict, so zero-area faces are never
 * picked and a draw exactly on a boundary goes to the next face). Binary search for that
 * first index; clamp to F - 1.
 *
 * *margin receives the distance of r to the nearer of the picked face's two CDF boundaries,
 * in units of A (a boundary at 0 or at 1 separates nothing and counts as infinitely far). */
int orc_pick_face(const double* cdf, int F, float r, double* margin) {
    const double A = cdf[F - 1];
    const double t = (double)r * A;
    int lo = 0, hi = F; /* invariant: answer in [lo, hi] */
    while (lo < hi) {
        int mid = lo + (hi - lo) / 2;
        if (cdf[mid] > t)
            hi = mid;
        else
            lo = mid + 1;
    }
    int f = lo < F ? lo : F - 1;
    if (margin) {
        double lower = f > 0 ? fabs((double)r - cdf[f - 1] / A) : INFINITY;
        double upper = f < F - 1 ? fabs(cdf[f] / A - (double)r) : INFINITY;
        *margin = lower < upper ? lower : upper;
    }
    return f;
}

/* Eq. 3 with the uniform-on-triangle reparameterisation (sqrt(r1), r2): the weights of the
 * face's vertices 0, 1, 2. They sum to 1. */
void orc_bary(float r1, float r2, double w[3]) {
    double s = sqrt((double)r1);
    w[0] = 1.0 - s;
    w[1] = s * (1.0 - (double)r2);
    w[2] = s * (double)r2;
}

/* The same point in float32, in the evaluation order stated at the top of the file. */
static void point_f32(const float* p0, const float* p1, const float* p2, float r1, float r2,
                      float x[3]) {
    float s = sqrtf(r1);
    float w0 = 1.0f - s;
    float w1 = s * (1.0f - r2);
    float w2 = s * r2;
    for (int k = 0; k < 3; ++k) x[k] = fmaf(w2, p2[k], fmaf(w1, p1[k], w0 * p0[k]));
}

/* Squared distance in float32, in the evaluation order stated at the top of the file. */
static float dist2_f32(const float* a, const float* b) {
    float dx = a[0] - b[0];
    float dy = a[1] - b[1];
    float dz = a[2] - b[2];
    return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

static double dist2_f64(const double* a, const double* b) {
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* Brute-force nearest neighbour of each of the n queries q among the m points p, decided in
 * float32: the first index with the smallest distance. best/second receive the smallest and
 * the second-smallest float32 distance (equal when the minimum is tied). */
static void nn_f32(const float* q, int n, const float* p, int m, int32_t* nn, float* best,
                   float* second) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        float b = INFINITY, s2 = INFINITY;
        int bi = -1;
        for (int j = 0; j < m; ++j) {
            float d = dist2_f32(q + 3 * (int64_t)i, p + 3 * (int64_t)j);
            if (d < b) {
                s2 = b;
                b = d;
                bi = j;
            } else if (d < s2) {
                s2 = d;
            }
        }
        nn[i] = bi;
        if (best) best[i] = b;
        if (second) second[i] = s2;
    }
}

/* The exact double-precision minimum distance of each query (used only to check that the
 * float32 decision changes the loss by no more than rounding). */
static void min_f64(const double* q, int n, const double* p, int m, double* best) {
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double b = INFINITY;
        for (int j = 0; j < m; ++j) {
            double d = dist2_f64(q + 3 * (int64_t)i, p + 3 * (int64_t)j);
            if (d < b) b = d;
        }
        best[i] = b;
    }
}

/*
 * One frame of the loss and its gradient.
 *   verts [V][3], faces [F][3] (0-based), draws [N][3] = (r_f, r1, r2), tgt [M][3].
 *   mask [F], nullable: sample only faces with a nonzero entry (orc_mask_areas).
 *   mode: ORC_BIDIR_MEAN (Eq. 1) or ORC_UNIDIR_SUM (Eq. 2).
 *   gscale: multiplier of dL_t in the gradient outputs (the upstream derivative).
 *   exact64: also compute loss_exact from the double-precision minima.
 * Every output pointer may be NULL. grad_verts, grad_points and grad_targets are overwritten.
 * Returns ORC_OK, ORC_EINVAL (empty sizes or a face index out of range) or ORC_EDEGENERATE
 * (total area zero or not finite).
 */
int orc_frame(const float* verts, const int32_t* faces, const uint8_t* mask, int V, int F,
              const float* draws, int N,
              const float* tgt, int M, int mode, double gscale, int exact64, double* loss,
              double* loss_exact, double* grad_verts, int32_t* face_idx, double* margin,
              double* bary, double* x64_out, float* x32_out, int32_t* nn_ab, float* d_ab,
              float* d2_ab, int32_t* nn_ba, float* d_ba, float* d2_ba, double* grad_points,
              double* grad_targets) {
    if (V <= 0 || F <= 0 || N <= 0 || M <= 0 || !verts || !faces || !draws || !tgt)
        return ORC_EINVAL;
    if (mode != ORC_BIDIR_MEAN && mode != ORC_UNIDIR_SUM) return ORC_EINVAL;
    for (int64_t k = 0; k < 3 * (int64_t)F; ++k)
        if (faces[k] < 0 || faces[k] >= V) return ORC_EINVAL;

    int rc = ORC_OK;
    double* area = malloc(sizeof(double) * F);
    double* cdf = malloc(sizeof(double) * F);
    int32_t* fi = malloc(sizeof(int32_t) * N);
    double* w = malloc(sizeof(double) * 3 * (size_t)N);
    double* x = malloc(sizeof(double) * 3 * (size_t)N);
    float* x32 = malloc(sizeof(float) * 3 * (size_t)N);
    double* y = malloc(sizeof(double) * 3 * (size_t)M);
    int32_t* ab = malloc(sizeof(int32_t) * N);
    int32_t* ba = malloc(sizeof(int32_t) * M);
    double* g = calloc(3 * (size_t)N, sizeof(double));

    orc_face_areas(verts, faces, F, area);
    if (mask) orc_mask_areas(area, mask, F);
    orc_area_cdf(area, F, cdf);
    const double A = cdf[F - 1];
    if (!(A > 0.0) || !isfinite(A)) {
        rc = ORC_EDEGENERATE;
        goto done;
    }

    /* sampling: face pick (Sec. III-B) and barycentric point (Eq. 3) */
    for (int i = 0; i < N; ++i) {
        const float* r = draws + 3 * (int64_t)i;
        double mg;
        int f = orc_pick_face(cdf, F, r[0], &mg);
        fi[i] = f;
        if (margin) margin[i] = mg;
        orc_bary(r[1], r[2], w + 3 * (int64_t)i);
        const float* p0 = verts + 3 * (int64_t)faces[3 * f + 0];
        const float* p1 = verts + 3 * (int64_t)faces[3 * f + 1];
        const float* p2 = verts + 3 * (int64_t)faces[3 * f + 2];
        for (int k = 0; k < 3; ++k)
            x[3 * i + k] = w[3 * i + 0] * p0[k] + w[3 * i + 1] * p1[k] + w[3 * i + 2] * p2[k];
        point_f32(p0, p1, p2, r[1], r[2], x32 + 3 * (int64_t)i);
    }
    for (int64_t k = 0; k < 3 * (int64_t)M; ++k) y[k] = (double)tgt[k];

    /* nearest neighbours (decided in float32), both directions for Eq. 1 */
    nn_f32(x32, N, tgt, M, ab, d_ab, d2_ab);
    if (mode == ORC_BIDIR_MEAN) nn_f32(tgt, M, x32, N, ba, d_ba, d2_ba);

    /* loss (Eq. 1 / Eq. 2) in double along the chosen neighbours */
    double s_ab = 0.0, s_ba = 0.0;
    for (int i = 0; i < N; ++i) s_ab += dist2_f64(x + 3 * (int64_t)i, y + 3 * (int64_t)ab[i]);
    if (mode == ORC_BIDIR_MEAN)
        for (int j = 0; j < M; ++j)
            s_ba += dist2_f64(y + 3 * (int64_t)j, x + 3 * (int64_t)ba[j]);
    double L = mode == ORC_BIDIR_MEAN ? s_ab / N + s_ba / M : s_ab;
    if (loss) *loss = L;

    if (exact64 && loss_exact) {
        double* bx = malloc(sizeof(double) * N);
        double* by = malloc(sizeof(double) * M);
        min_f64(x, N, y, M, bx);
        double ex = 0.0, ey = 0.0;
        for (int i = 0; i < N; ++i) ex += bx[i];
        if (mode == ORC_BIDIR_MEAN) {
            min_f64(y, M, x, N, by);
            for (int j = 0; j < M; ++j) ey += by[j];
        }
        *loss_exact = mode == ORC_BIDIR_MEAN ? ex / N + ey / M : ex;
        free(bx);
        free(by);
    }

    /* gradient of gscale * L_t with respect to the sampled points: d|x - y|^2/dx = 2 (x - y)
     * along the chosen neighbour, for each term of Eq. 1 / Eq. 2 */
    const double cab = mode == ORC_BIDIR_MEAN ? 2.0 * gscale / N : 2.0 * gscale;
    const double cba = 2.0 * gscale / M;
    if (grad_targets) memset(grad_targets, 0, sizeof(double) * 3 * (size_t)M);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < 3; ++k) {
            double t = cab * (x[3 * i + k] - y[3 * (int64_t)ab[i] + k]);
            g[3 * i + k] += t;
            if (grad_targets) grad_targets[3 * (int64_t)ab[i] + k] -= t;
        }
    if (mode == ORC_BIDIR_MEAN)
        for (int j = 0; j < M; ++j)
            for (int k = 0; k < 3; ++k) {
                double t = cba * (x[3 * (int64_t)ba[j] + k] - y[3 * (int64_t)j + k]);
                g[3 * (int64_t)ba[j] + k] += t;
                if (grad_targets) grad_targets[3 * (int64_t)j + k] -= t;
            }

    /* Eq. 4: dx_i/dp_{i,k} = w_{i,k}; the face pick is piecewise constant in the vertices and
     * contributes nothing. Scatter in point order. */
    if (grad_verts) {
        memset(grad_verts, 0, sizeof(double) * 3 * (size_t)V);
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) {
                int v = faces[3 * fi[i] + c];
                for (int k = 0; k < 3; ++k) grad_verts[3 * v + k] += w[3 * i + c] * g[3 * i + k];
            }
    }

    if (face_idx) memcpy(face_idx, fi, sizeof(int32_t) * N);
    if (bary) memcpy(bary, w, sizeof(double) * 3 * (size_t)N);
    if (x64_out) memcpy(x64_out, x, sizeof(double) * 3 * (size_t)N);
    if (x32_out) memcpy(x32_out, x32, sizeof(float) * 3 * (size_t)N);
    if (nn_ab) memcpy(nn_ab, ab, sizeof(int32_t) * N);
    if (nn_ba) {
        if (mode == ORC_BIDIR_MEAN)
            memcpy(nn_ba, ba, sizeof(int32_t) * M);
        else
            for (int j = 0; j < M; ++j) nn_ba[j] = -1;
    }
    if (grad_points) memcpy(grad_points, g, sizeof(double) * 3 * (size_t)N);

done:
    free(area);
    free(cdf);
    free(fi);
    free(w);
    free(x);
    free(x32);
    free(y);
    free(ab);
    free(ba);
    free(g);
    return rc;
}

/* Brute-force nearest neighbours of two given clouds in float32 (both directions), for the
 * Chamfer-only entry point: nn_ab [n], nn_ba [m], and the float32 minimum distances. */
void orc_nn_pair(const float* a, int n, const float* b, int m, int32_t* nn_ab, float* d_ab,
                 float* d2_ab, int32_t* nn_ba, float* d_ba, float* d2_ba) {
    nn_f32(a, n, b, m, nn_ab, d_ab, d2_ab);
    if (nn_ba) nn_f32(b, m, a, n, nn_ba, d_ba, d2_ba);
}

/* Chamfer loss of two given clouds (Eq. 1 or Eq. 2) in double, along float32-decided
 * neighbours, and its gradient with respect to the first cloud (overwritten, nullable). */
int orc_chamfer(const float* a, int n, const float* b, int m, int mode, double gscale,
                double* loss, double* grad_a) {
    if (n <= 0 || m <= 0) return ORC_EINVAL;
    int32_t* ab = malloc(sizeof(int32_t) * n);
    int32_t* ba = malloc(sizeof(int32_t) * m);
    nn_f32(a, n, b, m, ab, NULL, NULL);
    if (mode == ORC_BIDIR_MEAN) nn_f32(b, m, a, n, ba, NULL, NULL);
    double s_ab = 0.0, s_ba = 0.0;
    if (grad_a) memset(grad_a, 0, sizeof(double) * 3 * (size_t)n);
    const double cab = mode == ORC_BIDIR_MEAN ? 2.0 * gscale / n : 2.0 * gscale;
    const double cba = 2.0 * gscale / m;
    for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int k = 0; k < 3; ++k) {
            double t = (double)a[3 * i + k] - (double)b[3 * (int64_t)ab[i] + k];
            d += t * t;
            if (grad_a) grad_a[3 * i + k] += cab * t;
        }
        s_ab += d;
    }
    if (mode == ORC_BIDIR_MEAN)
        for (int j = 0; j < m; ++j) {
            double d = 0.0;
            for (int k = 0; k < 3; ++k) {
                double t = (double)a[3 * (int64_t)ba[j] + k] - (double)b[3 * j + k];
                d += t * t;
                if (grad_a) grad_a[3 * (int64_t)ba[j] + k] += cba * t;
            }
            s_ba += d;
        }
    *loss = mode == ORC_BIDIR_MEAN ? s_ab / n + s_ba / m : s_ab;
    free(ab);
    free(ba);
    return ORC_OK;
}
