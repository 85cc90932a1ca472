/*
 * hivc_oracle.c -- plain, slow FP64 CPU oracle for the decoder reconstruction
 * of "Inpainting-based Video Compression in FullHD" (Andris, Peter, Kaja
 * Mohideen, Weickert, Hoffmann; Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  The CUDA decoder shares no
 * code, header, table or constant with it.
 *
 * Every function states the passage it follows.  Readings of the paper where
 * it is silent (flow interpolation, block edge shapes, boundary type) are
 * listed next to the code that uses them.
 *
 * Image vectors are row-major (index y*W + x), as in Sec. 2.1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORACLE_OK 0
#define ORACLE_NOT_CONVERGED 1
#define ORACLE_INVALID (-1)
#define ORACLE_NOMEM (-2)

/* ========================================================================
 * Sec. 2.1, Eq. (1):  M (u - f) - (I - M) A u = 0  with  A = -L.
 *
 * L is the 5-point discrete Laplacian with reflecting boundary conditions:
 * a mirrored ghost pixel equals its inner neighbour, so a missing neighbour
 * contributes nothing:  (L u)_i = sum over in-image 4-neighbours j of
 * (u_j - u_i).  Grid size h = 1 (grey levels per pixel^2).
 * ======================================================================== */
static double laplace_at(const double *u, int W, int H, int x, int y)
{
    const double c = u[(size_t)y * W + x];
    double s = 0.0;
    if (x > 0) s += u[(size_t)y * W + x - 1] - c;
    if (x < W - 1) s += u[(size_t)y * W + x + 1] - c;
    if (y > 0) s += u[(size_t)(y - 1) * W + x] - c;
    if (y < H - 1) s += u[(size_t)(y + 1) * W + x] - c;
    return s;
}

/* max over unknown pixels of |(L u)_i|: the residual of Eq. (1). */
double oracle_inpaint_residual(int W, int H, const uint8_t *mask, const double *u)
{
    double m = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            if (!mask[(size_t)y * W + x]) {
                double r = fabs(laplace_at(u, W, H, x, y));
                if (r > m) m = r;
            }
    return m;
}

/* q = (-L) p restricted to unknown pixels, with p = 0 on the mask. */
static void apply_neg_laplace(const double *p, double *q, const uint8_t *mask, int W, int H)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            q[i] = mask[i] ? 0.0 : -laplace_at(p, W, H, x, y);
        }
}

/*
 * Homogeneous diffusion inpainting (Sec. 2.1, Eq. 1).
 *
 * u = f at the K mask pixels idx[] (values val[]), (L u)_i = 0 elsewhere.
 * On the unknown set U the system is  (-L_UU) u_U = L_UK f_K, symmetric
 * positive definite when K >= 1 (the grid is connected).  It is solved by
 * plain conjugate gradients started from the mean mask value, until the
 * true residual max_U |(L u)_i| <= tol.  The paper's coarse-to-fine cascade
 * only provides a better starting guess; the converged solution is the same.
 *
 * idx must be strictly increasing and < W*H; K >= 1.
 * Returns ORACLE_OK, ORACLE_NOT_CONVERGED (after max_iter iterations) or
 * ORACLE_INVALID.  *resid_out receives the final residual, *iters_out the
 * number of CG iterations.
 */
int oracle_inpaint(int W, int H, const uint32_t *idx, const double *val, int K,
                   double tol, int max_iter, double *u, double *resid_out, int *iters_out)
{
    const size_t N = (size_t)W * H;
    if (W < 1 || H < 1 || K < 1 || (size_t)K > N) return ORACLE_INVALID;
    for (int k = 0; k < K; ++k) {
        if (idx[k] >= N) return ORACLE_INVALID;
        if (k > 0 && idx[k] <= idx[k - 1]) return ORACLE_INVALID;
    }
    uint8_t *mask = (uint8_t *)calloc(N, 1);
    double *r = (double *)malloc(N * sizeof(double));
    double *p = (double *)malloc(N * sizeof(double));
    double *q = (double *)malloc(N * sizeof(double));
    if (!mask || !r || !p || !q) {
        free(mask); free(r); free(p); free(q);
        return ORACLE_NOMEM;
    }
    double mean = 0.0;
    for (int k = 0; k < K; ++k) { mask[idx[k]] = 1; mean += val[k]; }
    mean /= K;
    for (size_t i = 0; i < N; ++i) u[i] = mean;
    for (int k = 0; k < K; ++k) u[idx[k]] = val[k];

    int it = 0, status = ORACLE_NOT_CONVERGED;
    double res = 0.0;
    while (it < max_iter) {
        /* (re)start: r = b - (-L_UU) u_U = (L u)_U, p = r */
        double rr = 0.0;
        for (int y = 0; y < H; ++y)
            for (int x = 0; x < W; ++x) {
                size_t i = (size_t)y * W + x;
                r[i] = mask[i] ? 0.0 : laplace_at(u, W, H, x, y);
                p[i] = r[i];
                rr += r[i] * r[i];
            }
        res = 0.0;
        for (size_t i = 0; i < N; ++i) if (fabs(r[i]) > res) res = fabs(r[i]);
        if (res <= tol) { status = ORACLE_OK; break; }
        /* CG iterations until the recursive residual reaches tol, then the
           loop above recomputes the true residual. */
        int restart_at = it + 2000;
        while (it < max_iter && it < restart_at) {
            apply_neg_laplace(p, q, mask, W, H);
            double pq = 0.0;
            for (size_t i = 0; i < N; ++i) pq += p[i] * q[i];
            if (!(pq > 0.0)) break;
            double alpha = rr / pq, rr_new = 0.0, rmax = 0.0;
            for (size_t i = 0; i < N; ++i) {
                u[i] += alpha * p[i];
                r[i] -= alpha * q[i];
                rr_new += r[i] * r[i];
                if (fabs(r[i]) > rmax) rmax = fabs(r[i]);
            }
            ++it;
            if (rmax <= 0.25 * tol) break;
            double beta = rr_new / rr;
            rr = rr_new;
            for (size_t i = 0; i < N; ++i) p[i] = r[i] + beta * p[i];
        }
    }
    if (status != ORACLE_OK) {
        res = oracle_inpaint_residual(W, H, mask, u);
        if (res <= tol) status = ORACLE_OK;
    }
    /* mask pixels carry f exactly (Eq. 1, first term) */
    for (int k = 0; k < K; ++k) u[idx[k]] = val[k];
    if (resid_out) *resid_out = res;
    if (iters_out) *iters_out = it;
    free(mask); free(r); free(p); free(q);
    return status;
}

/* ========================================================================
 * Sec. 2 / 2.3: motion-compensated prediction along a backward optic flow
 * field.  pred(x) = ref(x + w(x)).  Reading: bilinear interpolation with the
 * sample position clamped to the plane (the paper does not state the
 * interpolation).
 * ======================================================================== */
static double bilinear_clamped(const double *ref, int W, int H, double X, double Y)
{
    double Xc = X < 0.0 ? 0.0 : (X > W - 1 ? (double)(W - 1) : X);
    double Yc = Y < 0.0 ? 0.0 : (Y > H - 1 ? (double)(H - 1) : Y);
    int x0 = (int)floor(Xc), y0 = (int)floor(Yc);
    if (x0 > W - 2) x0 = W - 2;
    if (y0 > H - 2) y0 = H - 2;
    if (x0 < 0) x0 = 0; /* W == 1 */
    if (y0 < 0) y0 = 0; /* H == 1 */
    double ax = Xc - x0, ay = Yc - y0;
    int x1 = x0 + 1 < W ? x0 + 1 : x0;
    int y1 = y0 + 1 < H ? y0 + 1 : y0;
    if (W == 1) ax = 0.0;
    if (H == 1) ay = 0.0;
    return (1 - ax) * (1 - ay) * ref[(size_t)y0 * W + x0]
         + ax * (1 - ay) * ref[(size_t)y0 * W + x1]
         + (1 - ax) * ay * ref[(size_t)y1 * W + x0]
         + ax * ay * ref[(size_t)y1 * W + x1];
}

/* Backward warp of one plane; flow is (dx, dy) per pixel, interleaved. */
void oracle_warp(int W, int H, const double *ref, const double *flow, double *pred)
{
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t i = (size_t)y * W + x;
            pred[i] = bilinear_clamped(ref, W, H, x + flow[2 * i], y + flow[2 * i + 1]);
        }
}

/*
 * Chroma flow for 4:2:0 planes (reading; the paper codes chroma at full
 * resolution after an RCT, Sec. 2.3): the chroma vector at (i, j) is half
 * the mean of the luma vectors of the in-plane pixels among
 * (2i..2i+1, 2j..2j+1).  Luma flow is float32 input (H x W x 2).
 */
void oracle_chroma_flow(int W, int H, const float *flow, int cw, int ch, double *flow_c)
{
    for (int j = 0; j < ch; ++j)
        for (int i = 0; i < cw; ++i) {
            double sx = 0.0, sy = 0.0;
            int n = 0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    int x = 2 * i + a, y = 2 * j + b;
                    if (x < W && y < H) {
                        sx += flow[2 * ((size_t)y * W + x)];
                        sy += flow[2 * ((size_t)y * W + x) + 1];
                        ++n;
                    }
                }
            flow_c[2 * ((size_t)j * cw + i)] = 0.5 * sx / n;
            flow_c[2 * ((size_t)j * cw + i) + 1] = 0.5 * sy / n;
        }
}

/* ========================================================================
 * Sec. 2.2: block-based pseudodifferential inpainting, harmonic operator.
 *
 * Each block is an independent w x h image with mirrored boundaries.  The
 * operator A = -L (Neumann, half-sample mirror) is diagonalised by the
 * orthonormal DCT-II (Eq. 4):  A phi_pq = mu_pq phi_pq  with
 *   phi_pq(x, y) = c_p(w) cos(pi p (2x+1) / 2w) * c_q(h) cos(pi q (2y+1) / 2h),
 *   c_0(n) = sqrt(1/n),  c_p(n) = sqrt(2/n),
 *   mu_pq = 4 sin^2(pi p / 2w) + 4 sin^2(pi q / 2h).
 * The Green's functions form the pseudo-inverse of A (Eqs. 2-3):
 *   G = sum_{(p,q) != (0,0)} phi_pq phi_pq^T / mu_pq .
 * ======================================================================== */
static double dct2_basis(int n, int p, int x)
{
    double c = (p == 0) ? sqrt(1.0 / n) : sqrt(2.0 / n);
    return c * cos(M_PI * p * (2.0 * x + 1.0) / (2.0 * n));
}

/* Eigenvalue of A = -L on the w x h block for mode (p, q). */
double oracle_block_eigenvalue(int w, int h, int p, int q)
{
    double sp = sin(M_PI * p / (2.0 * w)), sq = sin(M_PI * q / (2.0 * h));
    return 4.0 * sp * sp + 4.0 * sq * sq;
}

/*
 * G (N x N, N = w*h, pixel index y*w + x) from the eigen-expansion, for the
 * operator op (Sec. 2.2: the operator is defined by the eigenvalues of its
 * Green's functions and can be replaced):
 *   op 0: harmonic,    A = -L,     eigenvalues mu_pq,   G = sum phi phi^T / mu;
 *   op 1: biharmonic,  A = L^2,    eigenvalues mu_pq^2, G = sum phi phi^T / mu^2.
 * Both operators share the DCT-II eigenvectors and the constant null space.
 */
void oracle_green_matrix_op(int w, int h, int op, double *G)
{
    const int N = w * h;
    double *phi = (double *)malloc((size_t)N * sizeof(double));
    memset(G, 0, (size_t)N * N * sizeof(double));
    for (int q = 0; q < h; ++q)
        for (int p = 0; p < w; ++p) {
            if (p == 0 && q == 0) continue; /* null space of A: constants */
            const double mu = oracle_block_eigenvalue(w, h, p, q);
            double inv_mu = op == 1 ? 1.0 / (mu * mu) : 1.0 / mu;
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x)
                    phi[y * w + x] = dct2_basis(w, p, x) * dct2_basis(h, q, y);
            for (int i = 0; i < N; ++i) {
                double fi = phi[i] * inv_mu;
                for (int j = 0; j < N; ++j) G[(size_t)i * N + j] += fi * phi[j];
            }
        }
    free(phi);
}

/* The harmonic Green's matrix (op 0). */
void oracle_green_matrix(int w, int h, double *G) { oracle_green_matrix_op(w, h, 0, G); }

/* Dense LU with partial pivoting; solves S z = b in place (n x n, row-major).
   Returns 0, or -1 when a pivot is exactly zero. */
static int lu_solve(double *S, double *b, int n)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(S[(size_t)i * n + k]) > fabs(S[(size_t)piv * n + k])) piv = i;
        if (S[(size_t)piv * n + k] == 0.0) return -1;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = S[(size_t)k * n + j];
                S[(size_t)k * n + j] = S[(size_t)piv * n + j];
                S[(size_t)piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double l = S[(size_t)i * n + k] / S[(size_t)k * n + k];
            S[(size_t)i * n + k] = l;
            for (int j = k + 1; j < n; ++j) S[(size_t)i * n + j] -= l * S[(size_t)k * n + j];
            b[i] -= l * b[k];
        }
    }
    for (int k = n - 1; k >= 0; --k) {
        double s = b[k];
        for (int j = k + 1; j < n; ++j) s -= S[(size_t)k * n + j] * b[j];
        b[k] = s / S[(size_t)k * n + k];
    }
    return 0;
}

/*
 * One block (Sec. 2.2, Eqs. 2-3), given its Green's matrix G (w*h square).
 *
 * K = 0: r = 0 (zero data reconstructs as zero, Sec. 2.3).
 * K >= 1: the (K+1) x (K+1) system
 *     [ G_PP  1 ] [c]   [v]
 *     [ 1^T   0 ] [a] = [0]
 * (interpolation at the K points, coefficients summing to zero so that
 * A r = M c holds), solved by LU with partial pivoting; then
 *     r = G[:, P] c + a          (Eq. 3, explicit sum of Green's functions).
 * pos[] are point indices y*w + x, strictly increasing, K <= w*h - 1.
 * c_out (K values) and a_out may be NULL.
 */
int oracle_block_solve(int w, int h, const double *G, int K, const uint8_t *pos,
                       const double *v, double *r, double *c_out, double *a_out)
{
    const int N = w * h;
    if (K == 0) {
        for (int i = 0; i < N; ++i) r[i] = 0.0;
        if (a_out) *a_out = 0.0;
        return ORACLE_OK;
    }
    if (K > N - 1) return ORACLE_INVALID;
    for (int j = 0; j < K; ++j) {
        if (pos[j] >= N) return ORACLE_INVALID;
        if (j > 0 && pos[j] <= pos[j - 1]) return ORACLE_INVALID;
    }
    const int n = K + 1;
    double *S = (double *)malloc((size_t)n * n * sizeof(double));
    double *z = (double *)malloc((size_t)n * sizeof(double));
    for (int i = 0; i < K; ++i) {
        for (int j = 0; j < K; ++j) S[(size_t)i * n + j] = G[(size_t)pos[i] * N + pos[j]];
        S[(size_t)i * n + K] = 1.0;
        S[(size_t)K * n + i] = 1.0;
        z[i] = v[i];
    }
    S[(size_t)K * n + K] = 0.0;
    z[K] = 0.0;
    int st = lu_solve(S, z, n);
    if (st == 0) {
        const double a = z[K];
        for (int i = 0; i < N; ++i) {
            double s = a;
            for (int j = 0; j < K; ++j) s += z[j] * G[(size_t)i * N + pos[j]];
            r[i] = s;
        }
        if (c_out) for (int j = 0; j < K; ++j) c_out[j] = z[j];
        if (a_out) *a_out = a;
    }
    free(S); free(z);
    return st == 0 ? ORACLE_OK : ORACLE_INVALID;
}

/*
 * Residual plane from block data (Sec. 2.2, 2.3).  Blocks of edge B tile the
 * plane in raster order; edge blocks are cropped to the plane and treated as
 * independent images of their own size (reading: the paper uses 8 x 8 blocks
 * and does not discuss planes that are not multiples of 8).
 * block_ptr has nbx*nby + 1 entries; pos/val as in oracle_block_solve.
 * r is W x H.  Returns ORACLE_OK or ORACLE_INVALID (any bad block).
 */
int oracle_block_residual_op(int W, int H, int B, int op, const uint32_t *block_ptr,
                             const uint8_t *pos, const int16_t *val, double *r)
{
    if (W < 1 || H < 1 || B < 1 || B > 16) return ORACLE_INVALID;
    const int nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
    /* Green's matrices for the (at most four) block shapes of the plane */
    int shape_w[4], shape_h[4], n_shapes = 0;
    double *shape_G[4] = {0, 0, 0, 0};
    double *rb = (double *)malloc((size_t)B * B * sizeof(double));
    double *vb = (double *)malloc((size_t)B * B * sizeof(double));
    int status = ORACLE_OK;
    if (block_ptr[0] != 0) status = ORACLE_INVALID;
    for (int by = 0; by < nby && status == ORACLE_OK; ++by)
        for (int bx = 0; bx < nbx && status == ORACLE_OK; ++bx) {
            const int b = by * nbx + bx;
            const int w = (W - bx * B) < B ? (W - bx * B) : B;
            const int h = (H - by * B) < B ? (H - by * B) : B;
            if (block_ptr[b + 1] < block_ptr[b]) { status = ORACLE_INVALID; break; }
            const int K = (int)(block_ptr[b + 1] - block_ptr[b]);
            const uint8_t *pb = pos + block_ptr[b];
            double *G = NULL;
            for (int s = 0; s < n_shapes; ++s)
                if (shape_w[s] == w && shape_h[s] == h) G = shape_G[s];
            if (!G && K > 0) {
                G = (double *)malloc((size_t)w * h * w * h * sizeof(double));
                oracle_green_matrix_op(w, h, op, G);
                shape_w[n_shapes] = w; shape_h[n_shapes] = h; shape_G[n_shapes] = G;
                ++n_shapes;
            }
            for (int j = 0; j < K; ++j) vb[j] = val[block_ptr[b] + j];
            if (oracle_block_solve(w, h, G, K, pb, vb, rb, NULL, NULL) != ORACLE_OK) {
                status = ORACLE_INVALID;
                break;
            }
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x)
                    r[(size_t)(by * B + y) * W + bx * B + x] = rb[y * w + x];
        }
    for (int s = 0; s < n_shapes; ++s) free(shape_G[s]);
    free(rb); free(vb);
    return status;
}

/* The harmonic residual plane (op 0). */
int oracle_block_residual(int W, int H, int B, const uint32_t *block_ptr,
                          const uint8_t *pos, const int16_t *val, double *r)
{
    return oracle_block_residual_op(W, H, B, 0, block_ptr, pos, val, r);
}

/*
 * Coefficient mode (Sec. 2.2, 2.3): the decoder receives, per block, the
 * Green's coefficients of its points and the constant, and evaluates
 *     r = G[:, P] c + a                                   (Eq. 3)
 * without solving anything.  The coefficients arrive dead-zone quantised to
 * indices q in [-127, 127] (Sec. 2.3).  Reading (the mapping's scale is not
 * given): one quantiser step Delta per plane and a reconstruction offset
 * delta in [0, 1), as in the usual dead-zone scalar quantiser:
 *     c = 0 for q = 0,   c = sign(q) (|q| + delta) Delta  otherwise,
 * so that zero coefficients reconstruct as zero.  K = 0 gives r = a.
 * q = -128 is invalid.  pos as in oracle_block_solve (K <= w*h - 1).
 */
double oracle_dequantise(int q, double step, double offset)
{
    if (q == 0) return 0.0;
    const double m = (fabs((double)q) + offset) * step;
    return q < 0 ? -m : m;
}

int oracle_block_residual_coef(int W, int H, int B, int op, const uint32_t *block_ptr,
                               const uint8_t *pos, const int8_t *q, const float *a,
                               double step, double offset, double *r)
{
    if (W < 1 || H < 1 || B < 1 || B > 16) return ORACLE_INVALID;
    const int nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
    int shape_w[4], shape_h[4], n_shapes = 0;
    double *shape_G[4] = {0, 0, 0, 0};
    int status = ORACLE_OK;
    if (block_ptr[0] != 0) status = ORACLE_INVALID;
    for (int by = 0; by < nby && status == ORACLE_OK; ++by)
        for (int bx = 0; bx < nbx && status == ORACLE_OK; ++bx) {
            const int b = by * nbx + bx;
            const int w = (W - bx * B) < B ? (W - bx * B) : B;
            const int h = (H - by * B) < B ? (H - by * B) : B;
            const int N = w * h;
            if (block_ptr[b + 1] < block_ptr[b]) { status = ORACLE_INVALID; break; }
            const int K = (int)(block_ptr[b + 1] - block_ptr[b]);
            const uint8_t *pb = pos + block_ptr[b];
            const int8_t *qb = q + block_ptr[b];
            if (K > N - 1) { status = ORACLE_INVALID; break; }
            for (int j = 0; j < K; ++j)
                if (pb[j] >= N || (j > 0 && pb[j] <= pb[j - 1]) || qb[j] == -128) status = ORACLE_INVALID;
            if (status != ORACLE_OK) break;
            double *G = NULL;
            for (int s = 0; s < n_shapes; ++s)
                if (shape_w[s] == w && shape_h[s] == h) G = shape_G[s];
            if (!G && K > 0) {
                G = (double *)malloc((size_t)N * N * sizeof(double));
                oracle_green_matrix_op(w, h, op, G);
                shape_w[n_shapes] = w; shape_h[n_shapes] = h; shape_G[n_shapes] = G;
                ++n_shapes;
            }
            for (int y = 0; y < h; ++y)
                for (int x = 0; x < w; ++x) {
                    const int i = y * w + x;
                    double s = a[b];
                    for (int j = 0; j < K; ++j) s += oracle_dequantise(qb[j], step, offset) * G[(size_t)i * N + pb[j]];
                    r[(size_t)(by * B + y) * W + bx * B + x] = s;
                }
        }
    for (int s = 0; s < n_shapes; ++s) free(shape_G[s]);
    return status;
}

/*
 * Colour path of Sec. 2.3: the codec works on the planes of the reversible
 * colour transform (RCT) of JPEG2000 at full resolution (4:4:4):
 *     Y = floor((R + 2G + B) / 4),  U = B - G,  V = R - G,
 * so Y is in [0, 255] and U, V in [-255, 255].  The decoder's output is the
 * inverse transform of the rounded planes:
 *     G = Y - floor((U + V) / 4),  R = V + G,  B = U + G,
 * with each reconstructed plane first rounded half up to an integer
 * (reading: as for the uint8 planes) and R, G, B clamped to [0, 255].
 * y, u, v: n reconstructed values; rgb: 3 n bytes, planes R, G, B.
 */
void oracle_inverse_rct(int n, const double *y, const double *u, const double *v, uint8_t *rgb)
{
    for (int i = 0; i < n; ++i) {
        const double Y = floor(y[i] + 0.5), U = floor(u[i] + 0.5), V = floor(v[i] + 0.5);
        const double G = Y - floor((U + V) / 4.0);
        double c[3] = {V + G, G, U + G};
        for (int k = 0; k < 3; ++k) {
            const double x = c[k] < 0.0 ? 0.0 : (c[k] > 255.0 ? 255.0 : c[k]);
            rgb[(size_t)k * n + i] = (uint8_t)x;
        }
    }
}

/*
 * Side information by rectangular subdivision (Sec. 2.3: the BOFF is coded
 * as regions of a rectangular subdivision, each with its average value;
 * the mask points of every residual block come from a subdivision as
 * well).  The paper takes the subdivision from its reference [SPMEWB14]
 * and gives no bit format; the reading used here:
 *   - a node is a rectangle; a split halves its longer side (w >= h: the
 *     x side), the first part ceil(len/2), the second floor(len/2) long;
 *   - one bit per node in breadth-first order, 1 = split; a one-pixel
 *     node must carry 0; bits are packed LSB-first in 32-bit words;
 *   - leaves are numbered in breadth-first order;
 *   - a mask point is the centre pixel of its leaf,
 *     (x0 + (w-1)/2, y0 + (h-1)/2).
 */
static int tree_bit(const uint32_t *bits, long i) { return (int)((bits[i >> 5] >> (i & 31)) & 1u); }

/* Leaves (x0, y0, w, h per leaf, breadth-first) of the tree over the
   rectangle (x0, y0, w, h) whose bits are [b0, b0 + nbits).  Returns the
   number of bits used through *used, or ORACLE_INVALID (a split of a
   one-pixel node, bits exhausted, more than max_leaves leaves). */
int oracle_tree_leaves(int x0, int y0, int w, int h, const uint32_t *bits, long b0, long nbits, int *rects,
                       int max_leaves, int *n_leaves, long *used)
{
    int cap = 2 * w * h + 2;
    int *q = (int *)malloc((size_t)cap * 4 * sizeof(int));
    int head = 0, tail = 0, nl = 0, status = ORACLE_OK;
    long i = 0;
    q[0] = x0; q[1] = y0; q[2] = w; q[3] = h;
    tail = 1;
    while (head < tail) {
        const int *r = q + 4 * head++;
        if (i >= nbits) { status = ORACLE_INVALID; break; }
        const int split = tree_bit(bits, b0 + i++);
        if (!split) {
            if (nl >= max_leaves) { status = ORACLE_INVALID; break; }
            for (int k = 0; k < 4; ++k) rects[4 * nl + k] = r[k];
            ++nl;
            continue;
        }
        if (r[2] * r[3] < 2 || tail + 2 > cap) { status = ORACLE_INVALID; break; }
        int *a = q + 4 * tail, *b = q + 4 * (tail + 1);
        if (r[2] >= r[3]) {
            const int w1 = r[2] - r[2] / 2;
            a[0] = r[0]; a[1] = r[1]; a[2] = w1; a[3] = r[3];
            b[0] = r[0] + w1; b[1] = r[1]; b[2] = r[2] / 2; b[3] = r[3];
        } else {
            const int h1 = r[3] - r[3] / 2;
            a[0] = r[0]; a[1] = r[1]; a[2] = r[2]; a[3] = h1;
            b[0] = r[0]; b[1] = r[1] + h1; b[2] = r[2]; b[3] = r[3] / 2;
        }
        tail += 2;
    }
    free(q);
    *n_leaves = nl;
    *used = i;
    return status;
}

/* Dense backward flow (H x W x 2) from a subdivision tree over the plane
   and one (dx, dy) per leaf in breadth-first order.  The tree must use all
   nbits bits. */
int oracle_flow_from_tree(int W, int H, const uint32_t *bits, long nbits, const float *values, int n_values,
                          float *flow)
{
    int *rects = (int *)malloc((size_t)W * H * 4 * sizeof(int));
    int nl = 0;
    long used = 0;
    int st = oracle_tree_leaves(0, 0, W, H, bits, 0, nbits, rects, W * H, &nl, &used);
    if (st == ORACLE_OK && (used != nbits || nl != n_values)) st = ORACLE_INVALID;
    if (st == ORACLE_OK)
        for (int l = 0; l < nl; ++l) {
            const int *r = rects + 4 * l;
            for (int y = r[1]; y < r[1] + r[3]; ++y)
                for (int x = r[0]; x < r[0] + r[2]; ++x) {
                    flow[2 * ((size_t)y * W + x)] = values[2 * l];
                    flow[2 * ((size_t)y * W + x) + 1] = values[2 * l + 1];
                }
        }
    free(rects);
    return st;
}

static int cmp_u8(const void *a, const void *b) { return (int)*(const uint8_t *)a - (int)*(const uint8_t *)b; }

/* Residual mask positions of a plane's B x B blocks (raster order, edge
   blocks cropped) from one subdivision tree per block: block b's tree uses
   bits [tree_ptr[b], tree_ptr[b+1]) exactly.  Output as the residual data
   takes it: block_ptr (nblocks + 1) and pos (ly w + lx, increasing within
   a block), at most max_points points. */
int oracle_masks_from_trees(int W, int H, int B, const uint32_t *bits, const uint32_t *tree_ptr, uint32_t *block_ptr,
                            uint8_t *pos, long max_points)
{
    if (W < 1 || H < 1 || B < 1 || B > 16) return ORACLE_INVALID;
    const int nbx = (W + B - 1) / B, nby = (H + B - 1) / B;
    int rects[4 * 256];
    long n = 0;
    block_ptr[0] = 0;
    for (int b = 0; b < nbx * nby; ++b) {
        const int bx = b % nbx, by = b / nbx;
        const int w = (W - bx * B) < B ? (W - bx * B) : B;
        const int h = (H - by * B) < B ? (H - by * B) : B;
        if (tree_ptr[b + 1] < tree_ptr[b]) return ORACLE_INVALID;
        const long nb = (long)tree_ptr[b + 1] - tree_ptr[b];
        int nl = 0;
        long used = 0;
        if (oracle_tree_leaves(0, 0, w, h, bits, tree_ptr[b], nb, rects, 256, &nl, &used) != ORACLE_OK || used != nb)
            return ORACLE_INVALID;
        if (n + nl > max_points) return ORACLE_INVALID;
        for (int l = 0; l < nl; ++l) {
            const int *r = rects + 4 * l;
            pos[n + l] = (uint8_t)((r[1] + (r[3] - 1) / 2) * w + r[0] + (r[2] - 1) / 2);
        }
        qsort(pos + n, (size_t)nl, 1, cmp_u8);
        n += nl;
        block_ptr[b + 1] = (uint32_t)n;
    }
    return ORACLE_OK;
}

static int cmp_u32(const void *a, const void *b)
{
    const uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Intra mask positions (Sec. 2.3: the intra mask comes from a rectangular
   subdivision of the plane): the leaf centres of the plane's tree as sorted
   linear indices y W + x.  The tree must use all nbits bits. */
int oracle_intra_mask_from_tree(int W, int H, const uint32_t *bits, long nbits, uint32_t *idx, int *n)
{
    int *rects = (int *)malloc((size_t)W * H * 4 * sizeof(int));
    int nl = 0;
    long used = 0;
    int st = oracle_tree_leaves(0, 0, W, H, bits, 0, nbits, rects, W * H, &nl, &used);
    if (st == ORACLE_OK && used != nbits) st = ORACLE_INVALID;
    if (st == ORACLE_OK) {
        for (int l = 0; l < nl; ++l) {
            const int *r = rects + 4 * l;
            idx[l] = (uint32_t)(r[1] + (r[3] - 1) / 2) * (uint32_t)W + (uint32_t)(r[0] + (r[2] - 1) / 2);
        }
        qsort(idx, (size_t)nl, sizeof(uint32_t), cmp_u32);
        *n = nl;
    }
    free(rects);
    return st;
}
