/*
 * FP64 reference ("oracle") for efficient Bayesian multi-view deconvolution.
 *
 * TEST INFRASTRUCTURE ONLY. Only tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library. The CUDA product path never calls
 * it and shares no code with it.
 *
 * Everything here is written from the paper's equations, in plain loops and
 * FP64, in the order the paper states them:
 *   - single-view Richardson-Lucy update (Eq. 15) and its mirrored kernel
 *     (Suppl. Note "Integrating xi and x": integration over x is a
 *     convolution with P(-x));
 *   - convolution-algebra form of the multi-view update (Eq. 51);
 *   - compound kernel of the efficient method (Eq. 220, Eq. 222);
 *     optimization I (Eq. 230) and optimization II (Eq. 240);
 *   - sequential, view-by-view (OSEM-style) application of each view's
 *     update (Suppl. Note "Alternative iteration for faster convergence");
 *   - flat initial estimate equal to the mean observed intensity (Eq. 15 text);
 *   - reverse-mode gradient of K unrolled iterations (the paper does not
 *     differentiate its update; the chain rule through Eq. 15, Eq. 222 and the
 *     PSF normalisation of Eq. 3, pinned by FP64 central differences).
 *
 * Readings where the paper is silent (same on the CUDA side):
 *   - image convolutions are periodic (circular) on the given grid, i.e. what
 *     the Convolution Theorem computes; the zero and mirror boundaries are
 *     alternatives (mvdo_deconvolve_zero, mvdo_deconvolve_mirror);
 *   - kernel algebra (P_v^* * P_w * P_w^*) is linear convolution of the small
 *     kernels; the compound kernel lives on P_v's own box and is normalised
 *     to sum 1;
 *   - one floor eps: b <- max(b, eps) before the division and
 *     psi <- max(psi * c, eps) after the multiplication; default
 *     eps = 1e-4 * psi0;
 *   - psi0 is the mean over all voxels of all views.
 *
 * Layout: volumes are [z][y][x] (x fastest), dims = {X, Y, Z}. Kernels are
 * [Kz][Ky][Kx] with odd sizes; offset d = (i - (Kx-1)/2, ...) for index i.
 * Convolution: (f * k)(x) = sum_d k(d) f((x - d) mod dims).
 */
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#define MVDO_PLAIN 0
#define MVDO_EFFICIENT 1
#define MVDO_OPT1 2
#define MVDO_OPT2 3

static inline long idx3(int x, int y, int z, int X, int Y) { return (long)x + (long)X * ((long)y + (long)Y * z); }

int mvdo_num_threads(void) {
#ifdef _OPENMP
    int n = 1;
#pragma omp parallel
    {
#pragma omp single
        n = omp_get_num_threads();
    }
    return n;
#else
    return 1;
#endif
}

/* Periodic 3D convolution: out(x) = sum_d k(d) in((x - d) mod dims). */
void mvdo_conv(const double* in, const int dims[3], const double* k, const int kd[3], double* out) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const int Kx = kd[0], Ky = kd[1], Kz = kd[2];
    const int hx = (Kx - 1) / 2, hy = (Ky - 1) / 2, hz = (Kz - 1) / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Z; ++z) {
        for (int y = 0; y < Y; ++y) {
            double* o = out + idx3(0, y, z, X, Y);
            for (int x = 0; x < X; ++x) o[x] = 0.0;
            for (int kz = 0; kz < Kz; ++kz) {
                int sz = ((z - (kz - hz)) % Z + Z) % Z;
                for (int ky = 0; ky < Ky; ++ky) {
                    int sy = ((y - (ky - hy)) % Y + Y) % Y;
                    const double* src = in + idx3(0, sy, sz, X, Y);
                    const double* krow = k + (long)Kx * (ky + (long)Ky * kz);
                    for (int kx = 0; kx < Kx; ++kx) {
                        const double w = krow[kx];
                        const int dx = kx - hx; /* source index x - dx, wrapped */
                        if (dx >= 0) {
                            for (int x = 0; x < dx; ++x) o[x] += w * src[x - dx + X];
                            for (int x = dx; x < X; ++x) o[x] += w * src[x - dx];
                        } else {
                            for (int x = 0; x < X + dx; ++x) o[x] += w * src[x - dx];
                            for (int x = X + dx; x < X; ++x) o[x] += w * src[x - dx - X];
                        }
                    }
                }
            }
        }
    }
}

/* Mirrored kernel P^*(d) = P(-d) on the same centred box. */
void mvdo_mirror(const double* k, const int kd[3], double* out) {
    const int Kx = kd[0], Ky = kd[1], Kz = kd[2];
    for (int z = 0; z < Kz; ++z)
        for (int y = 0; y < Ky; ++y)
            for (int x = 0; x < Kx; ++x)
                out[idx3(Kx - 1 - x, Ky - 1 - y, Kz - 1 - z, Kx, Ky)] = k[idx3(x, y, z, Kx, Ky)];
}

/* Linear convolution of two small kernels, evaluated on a centred output box:
 * out(d) = sum_e a(e) b(d - e), with b taken as 0 outside its box. */
void mvdo_kconv(const double* a, const int ad[3], const double* b, const int bd[3],
                double* out, const int od[3]) {
    const int ahx = (ad[0] - 1) / 2, ahy = (ad[1] - 1) / 2, ahz = (ad[2] - 1) / 2;
    const int bhx = (bd[0] - 1) / 2, bhy = (bd[1] - 1) / 2, bhz = (bd[2] - 1) / 2;
    const int ohx = (od[0] - 1) / 2, ohy = (od[1] - 1) / 2, ohz = (od[2] - 1) / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int oz = 0; oz < od[2]; ++oz) {
        for (int oy = 0; oy < od[1]; ++oy) {
            for (int ox = 0; ox < od[0]; ++ox) {
                const int dx = ox - ohx, dy = oy - ohy, dz = oz - ohz;
                double s = 0.0;
                for (int ez = -ahz; ez <= ahz; ++ez) {
                    const int qz = dz - ez;
                    if (qz < -bhz || qz > bhz) continue;
                    for (int ey = -ahy; ey <= ahy; ++ey) {
                        const int qy = dy - ey;
                        if (qy < -bhy || qy > bhy) continue;
                        for (int ex = -ahx; ex <= ahx; ++ex) {
                            const int qx = dx - ex;
                            if (qx < -bhx || qx > bhx) continue;
                            s += a[idx3(ex + ahx, ey + ahy, ez + ahz, ad[0], ad[1])] *
                                 b[idx3(qx + bhx, qy + bhy, qz + bhz, bd[0], bd[1])];
                        }
                    }
                }
                out[idx3(ox, oy, oz, od[0], od[1])] = s;
            }
        }
    }
}

/* Kernel used for the back-projection of view v (the "compound" kernel).
 *   PLAIN:     P_v^*                                          (Eq. 51)
 *   EFFICIENT: P_v^* . prod_{w != v} (P_v^* * P_w * P_w^*)     (Eq. 220, Eq. 222)
 *   OPT1:      P_v^* . prod_{w != v} (P_v^* * P_w)             (Eq. 230)
 *   OPT2:      P_v^* . prod_{w != v} P_v^*  = (P_v^*)^N          (Eq. 240)
 * "." is the pointwise product on P_v's box; the result is normalised to sum 1.
 * Returns 0 on success, -1 if the result sums to 0. */
int mvdo_compound(int n_views, const double* const* psfs, const int* pdims /* n_views x 3 */,
                  int v, int variant, double* out) {
    const int* dv = pdims + 3 * v;
    const long Tv = (long)dv[0] * dv[1] * dv[2];
    double* pstar = (double*)malloc(sizeof(double) * Tv);
    double* cvw = (double*)malloc(sizeof(double) * Tv);
    mvdo_mirror(psfs[v], dv, pstar);
    for (long i = 0; i < Tv; ++i) out[i] = pstar[i];
    if (variant != MVDO_PLAIN) {
        for (int w = 0; w < n_views; ++w) {
            if (w == v) continue;
            const int* dw = pdims + 3 * w;
            if (variant == MVDO_EFFICIENT) {
                /* Q_w = P_w * P_w^*  on its full box (2K-1), then C_vw = P_v^* * Q_w on P_v's box */
                const long Tw = (long)dw[0] * dw[1] * dw[2];
                int qd[3] = {2 * dw[0] - 1, 2 * dw[1] - 1, 2 * dw[2] - 1};
                double* pwstar = (double*)malloc(sizeof(double) * Tw);
                double* q = (double*)malloc(sizeof(double) * (long)qd[0] * qd[1] * qd[2]);
                mvdo_mirror(psfs[w], dw, pwstar);
                mvdo_kconv(psfs[w], dw, pwstar, dw, q, qd);
                mvdo_kconv(pstar, dv, q, qd, cvw, dv);
                free(pwstar);
                free(q);
            } else if (variant == MVDO_OPT1) {
                mvdo_kconv(pstar, dv, psfs[w], dw, cvw, dv);
            } else { /* OPT2: P_w treated as constant, so the virtual factor is P_v^* itself */
                for (long i = 0; i < Tv; ++i) cvw[i] = pstar[i];
            }
            for (long i = 0; i < Tv; ++i) out[i] *= cvw[i];
        }
    }
    double s = 0.0;
    for (long i = 0; i < Tv; ++i) s += out[i];
    free(pstar);
    free(cvw);
    if (!(s > 0.0)) return -1;
    for (long i = 0; i < Tv; ++i) out[i] /= s;
    return 0;
}

/* One view update (a Richardson-Lucy step with kernel P and back-projection kernel K):
 *   b = psi * P ; r = phi / max(b, eps) ; c = r * K ; psi <- max(psi . c, eps).
 * b_out / r_out / c_out, when non-NULL, receive the intermediates. */
void mvdo_update(double* psi, const double* phi, const double* P, const int pd[3],
                 const double* K, const int kd[3], const int dims[3], double eps,
                 double* b_out, double* r_out, double* c_out) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double* b = b_out ? b_out : (double*)malloc(sizeof(double) * M);
    double* r = r_out ? r_out : (double*)malloc(sizeof(double) * M);
    double* c = c_out ? c_out : (double*)malloc(sizeof(double) * M);
    mvdo_conv(psi, dims, P, pd, b);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < M; ++i) r[i] = phi[i] / fmax(b[i], eps);
    mvdo_conv(r, dims, K, kd, c);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < M; ++i) psi[i] = fmax(psi[i] * c[i], eps);
    if (!b_out) free(b);
    if (!r_out) free(r);
    if (!c_out) free(c);
}

/* Mean over all voxels of all views (the flat initial estimate's value). */
double mvdo_mean_views(int n_views, const double* const* views, const int dims[3]) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double s = 0.0;
    for (int v = 0; v < n_views; ++v)
        for (long i = 0; i < M; ++i) s += views[v][i];
    return s / ((double)M * n_views);
}

/* Full deconvolution: PSFs normalised to sum 1, compound kernels, flat psi0
 * (unless init != 0, then psi holds the start), then n_iter iterations of the schedule (default 0..N-1),
 * each view's update applied to psi at once.
 * eps <= 0 selects 1e-4 * psi0. Returns the eps used, or -1 on error. */
double mvdo_deconvolve(int n_views, const double* const* views, const double* const* psfs,
                       const int* pdims, const int dims[3], int variant, int n_iter,
                       const int* schedule, int schedule_len, double eps, int init,
                       double* psi) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double psi0 = mvdo_mean_views(n_views, views, dims);
    if (eps <= 0.0) eps = 1e-4 * psi0;
    if (!init)
        for (long i = 0; i < M; ++i) psi[i] = psi0;
    /* every PSF is a probability distribution: normalise to sum 1 (Eq. 3) */
    double** pn = (double**)malloc(sizeof(double*) * n_views);
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) pn[v][i] = psfs[v][i] / s;
    }
    double** comp = (double**)malloc(sizeof(double*) * n_views);
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        comp[v] = (double*)malloc(sizeof(double) * T);
        if (mvdo_compound(n_views, (const double* const*)pn, pdims, v, variant, comp[v]) != 0) {
            for (int u = 0; u <= v; ++u) free(comp[u]);
            for (int u = 0; u < n_views; ++u) free(pn[u]);
            free(comp);
            free(pn);
            return -1.0;
        }
    }
    double* b = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* c = (double*)malloc(sizeof(double) * M);
    int L = (schedule && schedule_len > 0) ? schedule_len : n_views;
    for (int it = 0; it < n_iter; ++it) {
        for (int s = 0; s < L; ++s) {
            int v = (schedule && schedule_len > 0) ? schedule[s] : s;
            mvdo_update(psi, views[v], pn[v], pdims + 3 * v, comp[v], pdims + 3 * v, dims, eps, b, r, c);
        }
    }
    for (int v = 0; v < n_views; ++v) free(comp[v]);
    for (int v = 0; v < n_views; ++v) free(pn[v]);
    free(comp);
    free(pn);
    free(b);
    free(r);
    free(c);
    return eps;
}

/* Combined (simultaneous) update of Eq. 50 / Eq. 220: every view's factor
 *   c_v = (phi_v / max(psi * P_v, eps)) * K_v
 * is computed from the same psi, then psi <- max(psi . prod_v c_v, eps). With
 * root != 0 the product's |V|-th root is taken (the geometric mean of the
 * factors, as in the convergence proof, Section "Proof of convergence").
 * PSF normalisation, compound kernels, psi0 and eps as in mvdo_deconvolve.
 * Returns the eps used, or -1 on error. */
double mvdo_deconvolve_combined(int n_views, const double* const* views, const double* const* psfs,
                                const int* pdims, const int dims[3], int variant, int n_iter, int root,
                                double eps, int init, double* psi) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double psi0 = mvdo_mean_views(n_views, views, dims);
    if (eps <= 0.0) eps = 1e-4 * psi0;
    if (!init)
        for (long i = 0; i < M; ++i) psi[i] = psi0;
    double** pn = (double**)malloc(sizeof(double*) * n_views);
    double** comp = (double**)malloc(sizeof(double*) * n_views);
    int bad = 0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) pn[v][i] = psfs[v][i] / s;
    }
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        comp[v] = (double*)malloc(sizeof(double) * T);
        if (mvdo_compound(n_views, (const double* const*)pn, pdims, v, variant, comp[v]) != 0) bad = 1;
    }
    double* b = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* c = (double*)malloc(sizeof(double) * M);
    double* prod = (double*)malloc(sizeof(double) * M);
    for (int it = 0; it < n_iter && !bad; ++it) {
        for (long i = 0; i < M; ++i) prod[i] = 1.0;
        for (int v = 0; v < n_views; ++v) {
            const int* pd = pdims + 3 * v;
            mvdo_conv(psi, dims, pn[v], pd, b);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) r[i] = views[v][i] / fmax(b[i], eps);
            mvdo_conv(r, dims, comp[v], pd, c);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) prod[i] *= c[i];
        }
#pragma omp parallel for schedule(static)
        for (long i = 0; i < M; ++i) {
            const double f = root ? pow(prod[i], 1.0 / n_views) : prod[i];
            psi[i] = fmax(psi[i] * f, eps);
        }
    }
    for (int v = 0; v < n_views; ++v) {
        free(comp[v]);
        free(pn[v]);
    }
    free(comp);
    free(pn);
    free(b);
    free(r);
    free(c);
    free(prod);
    return bad ? -1.0 : eps;
}

/* Partially overlapping views (Suppl. Note "Partially overlapping datasets").
 * Each view carries a weight image w_v in [0, 1] (a blending function: 1 in
 * the view's central part, falling to 0 towards its boundary). Normalisation:
 * per voxel, with S = sum_v w_v, every weight is scaled by min(1, T / S), so
 * the sum is at most T and no weight ever grows; T is 1 (norm 0), the minimal
 * number of views overlapping at a voxel (norm 1), the average number (norm
 * 2), or `value` (norm 3). The number of views overlapping at a voxel counts
 * the views with w_v > 0; the minimum and the average run over the voxels at
 * least one view covers. Returns T, or -1 on a bad argument. */
double mvdo_normalize_weights(int n_views, const double* const* w, const int dims[3], int norm, double value,
                              double* const* out) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double T = 1.0;
    if (norm == 1 || norm == 2) {
        long covered = 0, sum = 0;
        int mn = n_views + 1;
        for (long i = 0; i < M; ++i) {
            int n = 0;
            for (int v = 0; v < n_views; ++v) n += w[v][i] > 0.0;
            if (n == 0) continue;
            ++covered;
            sum += n;
            if (n < mn) mn = n;
        }
        if (covered == 0) return -1.0;
        T = norm == 1 ? (double)mn : (double)sum / (double)covered;
    } else if (norm == 3) {
        if (!(value > 0.0)) return -1.0;
        T = value;
    } else if (norm != 0) {
        return -1.0;
    }
    for (long i = 0; i < M; ++i) {
        double S = 0.0;
        for (int v = 0; v < n_views; ++v) S += w[v][i];
        const double f = S > T ? T / S : 1.0;
        for (int v = 0; v < n_views; ++v) out[v][i] = w[v][i] * f;
    }
    return T;
}

/* Sequential deconvolution with (already normalised) view weights and an
 * optional Tikhonov regularisation. The paper applies Tikhonov regularisation
 * (lambda) without printing its update; this oracle takes the one-step-late
 * MAP-EM of P. J. Green (IEEE Trans. Med. Imaging 9, 1990) with the quadratic
 * prior lambda/2 |psi|^2, whose factor for a view is f_v = c_v / (1 + lambda psi).
 * Each view update applies the fraction w_v of that change:
 *   psi <- max(psi + w_v (psi f_v - psi), eps) = max(psi (1 + w_v (f_v - 1)), eps).
 * weights == NULL means w_v = 1. Otherwise as mvdo_deconvolve (default
 * schedule). Returns eps, or -1. */
double mvdo_deconvolve_weighted(int n_views, const double* const* views, const double* const* psfs,
                                const int* pdims, const int dims[3], int variant, int n_iter,
                                const double* const* weights, double lambda, double eps, int init, double* psi) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double psi0 = mvdo_mean_views(n_views, views, dims);
    if (eps <= 0.0) eps = 1e-4 * psi0;
    if (!init)
        for (long i = 0; i < M; ++i) psi[i] = psi0;
    double** pn = (double**)malloc(sizeof(double*) * n_views);
    double** comp = (double**)malloc(sizeof(double*) * n_views);
    int bad = 0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) pn[v][i] = psfs[v][i] / s;
    }
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        comp[v] = (double*)malloc(sizeof(double) * T);
        if (mvdo_compound(n_views, (const double* const*)pn, pdims, v, variant, comp[v]) != 0) bad = 1;
    }
    double* b = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* c = (double*)malloc(sizeof(double) * M);
    for (int it = 0; it < n_iter && !bad; ++it) {
        for (int v = 0; v < n_views; ++v) {
            const int* pd = pdims + 3 * v;
            mvdo_conv(psi, dims, pn[v], pd, b);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) r[i] = views[v][i] / fmax(b[i], eps);
            mvdo_conv(r, dims, comp[v], pd, c);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) {
                const double f = c[i] / (1.0 + lambda * psi[i]);
                const double w = weights ? weights[v][i] : 1.0;
                psi[i] = fmax(psi[i] + w * (psi[i] * f - psi[i]), eps);
            }
        }
    }
    for (int v = 0; v < n_views; ++v) {
        free(comp[v]);
        free(pn[v]);
    }
    free(comp);
    free(pn);
    free(b);
    free(r);
    free(c);
    return bad ? -1.0 : eps;
}

/* Convolution with a zero boundary (the volume continued by zeros):
 *   out(x) = sum_d k(d) in(x - d), terms with x - d outside the grid dropped. */
void mvdo_conv_zero(const double* in, const int dims[3], const double* k, const int kd[3], double* out) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const int hx = (kd[0] - 1) / 2, hy = (kd[1] - 1) / 2, hz = (kd[2] - 1) / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                double s = 0.0;
                for (int tz = 0; tz < kd[2]; ++tz) {
                    const int sz = z - (tz - hz);
                    if (sz < 0 || sz >= Z) continue;
                    for (int ty = 0; ty < kd[1]; ++ty) {
                        const int sy = y - (ty - hy);
                        if (sy < 0 || sy >= Y) continue;
                        for (int tx = 0; tx < kd[0]; ++tx) {
                            const int sx = x - (tx - hx);
                            if (sx < 0 || sx >= X) continue;
                            s += k[tx + kd[0] * (ty + kd[1] * tz)] * in[idx3(sx, sy, sz, X, Y)];
                        }
                    }
                }
                out[idx3(x, y, z, X, Y)] = s;
            }
}

/* Sequential deconvolution (default schedule) with zero-boundary image
 * convolutions: b = psi * P_v and the back-projection r * P_v^comp treat the
 * volume as surrounded by zeros. The paper's convolutions are periodic; for
 * this forward model the update is the ML-EM step of Shepp and Vardi (1982),
 * which divides the back-projection by the sensitivity s_v = 1 * P_v^comp
 * (the back-projection of a field of ones, 1 in the periodic case):
 *   psi <- max(psi (r * P_v^comp) / s_v, eps).
 * With view weights w_v (NULL: none) and Tikhonov lambda the factor
 * f = ((r * P_v^comp) / s_v) / (1 + lambda psi) enters as in
 * mvdo_deconvolve_weighted: psi <- max(psi + w (psi f - psi), eps).
 * Otherwise as mvdo_deconvolve. Returns eps, or -1. */
double mvdo_deconvolve_zero(int n_views, const double* const* views, const double* const* psfs, const int* pdims,
                            const int dims[3], int variant, int n_iter, const double* const* weights, double lambda,
                            double eps, int init, double* psi) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double psi0 = mvdo_mean_views(n_views, views, dims);
    if (eps <= 0.0) eps = 1e-4 * psi0;
    if (!init)
        for (long i = 0; i < M; ++i) psi[i] = psi0;
    double** pn = (double**)malloc(sizeof(double*) * n_views);
    double** comp = (double**)malloc(sizeof(double*) * n_views);
    int bad = 0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) pn[v][i] = psfs[v][i] / s;
    }
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        comp[v] = (double*)malloc(sizeof(double) * T);
        if (mvdo_compound(n_views, (const double* const*)pn, pdims, v, variant, comp[v]) != 0) bad = 1;
    }
    double* b = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* c = (double*)malloc(sizeof(double) * M);
    double* ones = (double*)malloc(sizeof(double) * M);
    double** sens = (double**)malloc(sizeof(double*) * n_views);
    for (long i = 0; i < M; ++i) ones[i] = 1.0;
    for (int v = 0; v < n_views; ++v) {
        sens[v] = (double*)malloc(sizeof(double) * M);
        if (!bad) mvdo_conv_zero(ones, dims, comp[v], pdims + 3 * v, sens[v]);
    }
    for (int it = 0; it < n_iter && !bad; ++it) {
        for (int v = 0; v < n_views; ++v) {
            const int* pd = pdims + 3 * v;
            mvdo_conv_zero(psi, dims, pn[v], pd, b);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) r[i] = views[v][i] / fmax(b[i], eps);
            mvdo_conv_zero(r, dims, comp[v], pd, c);
            if (!weights && lambda == 0.0) {
#pragma omp parallel for schedule(static)
                for (long i = 0; i < M; ++i) psi[i] = fmax(psi[i] * c[i] / sens[v][i], eps);
            } else {
#pragma omp parallel for schedule(static)
                for (long i = 0; i < M; ++i) {
                    const double f = c[i] / sens[v][i] / (1.0 + lambda * psi[i]);
                    const double w = weights ? weights[v][i] : 1.0;
                    psi[i] = fmax(psi[i] + w * (psi[i] * f - psi[i]), eps);
                }
            }
        }
    }
    for (int v = 0; v < n_views; ++v) {
        free(comp[v]);
        free(pn[v]);
        free(sens[v]);
    }
    free(comp);
    free(pn);
    free(sens);
    free(ones);
    free(b);
    free(r);
    free(c);
    return bad ? -1.0 : eps;
}

/* Half-sample symmetric reflection of index i into [0, n): the grid continued
 * as ... x1 x0 | x0 x1 ... x(n-1) | x(n-1) x(n-2) ... (period 2n). */
static int reflect(int i, int n) {
    int m = i % (2 * n);
    if (m < 0) m += 2 * n;
    return m < n ? m : 2 * n - 1 - m;
}

/* Convolution with a mirror boundary (the volume continued by reflection):
 *   out(x) = sum_d k(d) in(reflect(x - d)). */
void mvdo_conv_mirror(const double* in, const int dims[3], const double* k, const int kd[3], double* out) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const int hx = (kd[0] - 1) / 2, hy = (kd[1] - 1) / 2, hz = (kd[2] - 1) / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                double s = 0.0;
                for (int tz = 0; tz < kd[2]; ++tz) {
                    const int sz = reflect(z - (tz - hz), Z);
                    for (int ty = 0; ty < kd[1]; ++ty) {
                        const int sy = reflect(y - (ty - hy), Y);
                        for (int tx = 0; tx < kd[0]; ++tx)
                            s += k[tx + kd[0] * (ty + kd[1] * tz)] * in[idx3(reflect(x - (tx - hx), X), sy, sz, X, Y)];
                    }
                }
                out[idx3(x, y, z, X, Y)] = s;
            }
}

/* Back-projection with a mirror boundary: each voxel i spreads r(i) k(e) to
 * i + e, and what lands outside the grid is folded back onto its reflection:
 *   out(j) = sum_i r(i) sum_{e : reflect(i + e) = j} k(e).
 * It is the transpose of mvdo_conv_mirror with the mirrored kernel k(-e), and
 * equals r * k when nothing reaches a face. Serial scatter. */
void mvdo_backproject_mirror(const double* r, const int dims[3], const double* k, const int kd[3], double* out) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const int hx = (kd[0] - 1) / 2, hy = (kd[1] - 1) / 2, hz = (kd[2] - 1) / 2;
    const long M = (long)X * Y * Z;
    for (long i = 0; i < M; ++i) out[i] = 0.0;
    for (int z = 0; z < Z; ++z)
        for (int y = 0; y < Y; ++y)
            for (int x = 0; x < X; ++x) {
                const double ri = r[idx3(x, y, z, X, Y)];
                for (int tz = 0; tz < kd[2]; ++tz) {
                    const int jz = reflect(z + (tz - hz), Z);
                    for (int ty = 0; ty < kd[1]; ++ty) {
                        const int jy = reflect(y + (ty - hy), Y);
                        for (int tx = 0; tx < kd[0]; ++tx)
                            out[idx3(reflect(x + (tx - hx), X), jy, jz, X, Y)] += ri * k[tx + kd[0] * (ty + kd[1] * tz)];
                    }
                }
            }
}

/* Sequential deconvolution (default schedule) with mirror-boundary image
 * convolutions. The forward blur is b = P_v convolved with the reflected
 * continuation of psi (mvdo_conv_mirror); the back-projection with P_v^comp
 * is the folded one (mvdo_backproject_mirror), which for the plain kernel
 * P_v^* is the exact transpose of the forward blur. As for the zero boundary,
 * the update is the ML-EM step that divides by the sensitivity s_v (the
 * back-projection of a field of ones; 1 wherever P_v^comp is symmetric under
 * the reflection of each face it reaches):
 *   psi <- max(psi c / s_v, eps),  c = backproject_mirror(r, P_v^comp).
 * View weights and Tikhonov lambda enter as in mvdo_deconvolve_zero.
 * Otherwise as mvdo_deconvolve. Returns eps, or -1. */
double mvdo_deconvolve_mirror(int n_views, const double* const* views, const double* const* psfs, const int* pdims,
                              const int dims[3], int variant, int n_iter, const double* const* weights,
                              double lambda, double eps, int init, double* psi) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double psi0 = mvdo_mean_views(n_views, views, dims);
    if (eps <= 0.0) eps = 1e-4 * psi0;
    if (!init)
        for (long i = 0; i < M; ++i) psi[i] = psi0;
    double** pn = (double**)malloc(sizeof(double*) * n_views);
    double** comp = (double**)malloc(sizeof(double*) * n_views);
    double** sens = (double**)malloc(sizeof(double*) * n_views);
    int bad = 0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) pn[v][i] = psfs[v][i] / s;
    }
    double* b = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* c = (double*)malloc(sizeof(double) * M);
    for (long i = 0; i < M; ++i) r[i] = 1.0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        comp[v] = (double*)malloc(sizeof(double) * T);
        sens[v] = (double*)malloc(sizeof(double) * M);
        if (mvdo_compound(n_views, (const double* const*)pn, pdims, v, variant, comp[v]) != 0) bad = 1;
        if (!bad) mvdo_backproject_mirror(r, dims, comp[v], pdims + 3 * v, sens[v]);
    }
    for (int it = 0; it < n_iter && !bad; ++it) {
        for (int v = 0; v < n_views; ++v) {
            const int* pd = pdims + 3 * v;
            mvdo_conv_mirror(psi, dims, pn[v], pd, b);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) r[i] = views[v][i] / fmax(b[i], eps);
            mvdo_backproject_mirror(r, dims, comp[v], pd, c);
            if (!weights && lambda == 0.0) {
#pragma omp parallel for schedule(static)
                for (long i = 0; i < M; ++i) psi[i] = fmax(psi[i] * c[i] / sens[v][i], eps);
            } else {
#pragma omp parallel for schedule(static)
                for (long i = 0; i < M; ++i) {
                    const double f = c[i] / sens[v][i] / (1.0 + lambda * psi[i]);
                    const double w = weights ? weights[v][i] : 1.0;
                    psi[i] = fmax(psi[i] + w * (psi[i] * f - psi[i]), eps);
                }
            }
        }
    }
    for (int v = 0; v < n_views; ++v) {
        free(comp[v]);
        free(pn[v]);
        free(sens[v]);
    }
    free(comp);
    free(pn);
    free(sens);
    free(b);
    free(r);
    free(c);
    return bad ? -1.0 : eps;
}

/* The combined update (as mvdo_deconvolve_combined) with a zero (boundary 1)
 * or mirror (boundary 2) boundary: every view's factor is its back-projected
 * ratio divided by its sensitivity, c_v / s_v (the blur and back-projection of
 * mvdo_deconvolve_zero or mvdo_deconvolve_mirror), and psi <- max(psi .
 * prod_v (c_v / s_v)^e, eps) with e = 1 / |V| when root != 0, else 1.
 * Returns eps, or -1 (also for an unknown boundary). */
double mvdo_deconvolve_combined_bounded(int n_views, const double* const* views, const double* const* psfs,
                                        const int* pdims, const int dims[3], int variant, int n_iter, int root,
                                        int boundary, double eps, int init, double* psi) {
    if (boundary != 1 && boundary != 2) return -1.0;
    const long M = (long)dims[0] * dims[1] * dims[2];
    double psi0 = mvdo_mean_views(n_views, views, dims);
    if (eps <= 0.0) eps = 1e-4 * psi0;
    if (!init)
        for (long i = 0; i < M; ++i) psi[i] = psi0;
    double** pn = (double**)malloc(sizeof(double*) * n_views);
    double** comp = (double**)malloc(sizeof(double*) * n_views);
    double** sens = (double**)malloc(sizeof(double*) * n_views);
    int bad = 0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) pn[v][i] = psfs[v][i] / s;
    }
    double* b = (double*)malloc(sizeof(double) * M);
    double* r = (double*)malloc(sizeof(double) * M);
    double* c = (double*)malloc(sizeof(double) * M);
    double* prod = (double*)malloc(sizeof(double) * M);
    for (long i = 0; i < M; ++i) r[i] = 1.0;
    for (int v = 0; v < n_views; ++v) {
        const long T = (long)pdims[3 * v] * pdims[3 * v + 1] * pdims[3 * v + 2];
        comp[v] = (double*)malloc(sizeof(double) * T);
        sens[v] = (double*)malloc(sizeof(double) * M);
        if (mvdo_compound(n_views, (const double* const*)pn, pdims, v, variant, comp[v]) != 0) bad = 1;
        if (bad) continue;
        if (boundary == 1)
            mvdo_conv_zero(r, dims, comp[v], pdims + 3 * v, sens[v]);
        else
            mvdo_backproject_mirror(r, dims, comp[v], pdims + 3 * v, sens[v]);
    }
    for (int it = 0; it < n_iter && !bad; ++it) {
        for (long i = 0; i < M; ++i) prod[i] = 1.0;
        for (int v = 0; v < n_views; ++v) {
            const int* pd = pdims + 3 * v;
            if (boundary == 1)
                mvdo_conv_zero(psi, dims, pn[v], pd, b);
            else
                mvdo_conv_mirror(psi, dims, pn[v], pd, b);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) r[i] = views[v][i] / fmax(b[i], eps);
            if (boundary == 1)
                mvdo_conv_zero(r, dims, comp[v], pd, c);
            else
                mvdo_backproject_mirror(r, dims, comp[v], pd, c);
#pragma omp parallel for schedule(static)
            for (long i = 0; i < M; ++i) prod[i] *= c[i] / sens[v][i];
        }
#pragma omp parallel for schedule(static)
        for (long i = 0; i < M; ++i) {
            const double f = root ? pow(prod[i], 1.0 / n_views) : prod[i];
            psi[i] = fmax(psi[i] * f, eps);
        }
    }
    for (int v = 0; v < n_views; ++v) {
        free(comp[v]);
        free(pn[v]);
        free(sens[v]);
    }
    free(comp);
    free(pn);
    free(sens);
    free(b);
    free(r);
    free(c);
    free(prod);
    return bad ? -1.0 : eps;
}

/* One view update evaluated only at the listed voxels (flat indices):
 *   out[i] = max(psi(x_i) * c(x_i), eps), with c, r, b computed from the
 * definitions above on the neighbourhood each sample needs. */
void mvdo_update_at(const double* psi, const double* phi, const double* P, const int pd[3],
                    const double* K, const int kd[3], const int dims[3], double eps,
                    const long* sample, int n_samples, double* out) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const int phx = (pd[0] - 1) / 2, phy = (pd[1] - 1) / 2, phz = (pd[2] - 1) / 2;
    const int khx = (kd[0] - 1) / 2, khy = (kd[1] - 1) / 2, khz = (kd[2] - 1) / 2;
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < n_samples; ++s) {
        const long li = sample[s];
        const int x = (int)(li % X), y = (int)((li / X) % Y), z = (int)(li / ((long)X * Y));
        double c = 0.0;
        for (int kz = 0; kz < kd[2]; ++kz)
            for (int ky = 0; ky < kd[1]; ++ky)
                for (int kx = 0; kx < kd[0]; ++kx) {
                    /* r at u = x - d */
                    const int ux = ((x - (kx - khx)) % X + X) % X;
                    const int uy = ((y - (ky - khy)) % Y + Y) % Y;
                    const int uz = ((z - (kz - khz)) % Z + Z) % Z;
                    double b = 0.0;
                    for (int pz = 0; pz < pd[2]; ++pz)
                        for (int py = 0; py < pd[1]; ++py)
                            for (int px = 0; px < pd[0]; ++px) {
                                const int sx = ((ux - (px - phx)) % X + X) % X;
                                const int sy = ((uy - (py - phy)) % Y + Y) % Y;
                                const int sz = ((uz - (pz - phz)) % Z + Z) % Z;
                                b += P[idx3(px, py, pz, pd[0], pd[1])] * psi[idx3(sx, sy, sz, X, Y)];
                            }
                    const double r = phi[idx3(ux, uy, uz, X, Y)] / fmax(b, eps);
                    c += K[idx3(kx, ky, kz, kd[0], kd[1])] * r;
                }
        out[s] = fmax(psi[li] * c, eps);
    }
}

/* ------------------------------------------------------------------------
 * Gradient of the unrolled iteration (reverse mode, FP64).
 *
 * Loss: L = mean_x (psi_K(x) - truth(x))^2 after n_iter iterations of the
 * schedule from the flat start psi0 = mean of the views. One update, written
 * as a chain of elementary steps (floors inactive where the derivative is
 * taken: max(a, eps) passes its gradient when a > eps, else none):
 *   b = psi * P ; b' = max(b, eps) ; r = phi / b' ; c = r * K ;
 *   t = psi . c ; psi' = max(t, eps)
 * and its adjoint, for an incoming gradient g = dL/dpsi':
 *   tb = g [t > eps] ; psi_bar = tb . c ; cb = tb . psi
 *   rb = cb * K^*            (K^*(d) = K(-d): transpose of the convolution)
 *   Kb(d) += sum_x cb(x) r(x - d)
 *   phib += rb / b' ; bb = -rb r / b' [b > eps]
 *   psi_bar += bb * P^* ; Pb(d) += sum_x bb(x) psi(x - d)
 * The kernel gradients Kb flow back through the compound kernel (Eq. 222,
 * 230 or 240 and the normalisation) to every PSF, the PSF gradients through
 * the PSF normalisation to the raw PSF values, and the gradient of psi0
 * (flat start = mean of all views) spreads evenly over every view voxel.
 * The floor eps = 1e-4 psi0 also depends on the views; it only acts through
 * active floors, which the gradient ignores as stated above.
 * ------------------------------------------------------------------------ */

/* out(d) = sum_x a(x) b((x - d) mod dims) for d on a centred box */
static void corr_box(const double* a, const double* b, const int dims[3], const int kd[3], double* out) {
    const int X = dims[0], Y = dims[1], Z = dims[2];
    const int hx = (kd[0] - 1) / 2, hy = (kd[1] - 1) / 2, hz = (kd[2] - 1) / 2;
    const long T = (long)kd[0] * kd[1] * kd[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (long i = 0; i < T; ++i) {
        const int dx = (int)(i % kd[0]) - hx, dy = (int)((i / kd[0]) % kd[1]) - hy,
                  dz = (int)(i / ((long)kd[0] * kd[1])) - hz;
        double s = 0.0;
        for (int z = 0; z < Z; ++z) {
            const int sz = ((z - dz) % Z + Z) % Z;
            for (int y = 0; y < Y; ++y) {
                const int sy = ((y - dy) % Y + Y) % Y;
                const double* ar = a + idx3(0, y, z, X, Y);
                const double* br = b + idx3(0, sy, sz, X, Y);
                for (int x = 0; x < X; ++x) s += ar[x] * br[((x - dx) % X + X) % X];
            }
        }
        out[i] = s;
    }
}

/* value of a centred-box kernel at offset (dx,dy,dz), 0 outside the box */
static double kat(const double* k, const int kd[3], int dx, int dy, int dz) {
    const int hx = (kd[0] - 1) / 2, hy = (kd[1] - 1) / 2, hz = (kd[2] - 1) / 2;
    if (dx < -hx || dx > hx || dy < -hy || dy > hy || dz < -hz || dz > hz) return 0.0;
    return k[idx3(dx + hx, dy + hy, dz + hz, kd[0], kd[1])];
}

/* Gradient of the compound kernel of view v (normalised PSFs Pn) with
 * respect to every normalised PSF: adds into Pb[w] given Kb (box of v). */
static void compound_vjp(int nv, double* const* Pn, const int* pd, int v, int variant, const double* Kb,
                         double* const* Pb) {
    const int* dv = pd + 3 * v;
    const long Tv = (long)dv[0] * dv[1] * dv[2];
    const int hvx = (dv[0] - 1) / 2, hvy = (dv[1] - 1) / 2, hvz = (dv[2] - 1) / 2;
    double* A = (double*)malloc(sizeof(double) * Tv);
    mvdo_mirror(Pn[v], dv, A);
    /* forward factors C_w on v's box (1 for w == v) */
    double** C = (double**)calloc(nv, sizeof(double*));
    double** Q = (double**)calloc(nv, sizeof(double*));
    int (*qd)[3] = malloc(sizeof(int[3]) * nv);
    double* U = (double*)malloc(sizeof(double) * Tv);
    for (long i = 0; i < Tv; ++i) U[i] = A[i];
    if (variant != MVDO_PLAIN) {
        for (int w = 0; w < nv; ++w) {
            if (w == v) continue;
            const int* dw = pd + 3 * w;
            C[w] = (double*)malloc(sizeof(double) * Tv);
            if (variant == MVDO_EFFICIENT) {
                const long Tw = (long)dw[0] * dw[1] * dw[2];
                qd[w][0] = 2 * dw[0] - 1;
                qd[w][1] = 2 * dw[1] - 1;
                qd[w][2] = 2 * dw[2] - 1;
                double* pws = (double*)malloc(sizeof(double) * Tw);
                Q[w] = (double*)malloc(sizeof(double) * (long)qd[w][0] * qd[w][1] * qd[w][2]);
                mvdo_mirror(Pn[w], dw, pws);
                mvdo_kconv(Pn[w], dw, pws, dw, Q[w], qd[w]);
                mvdo_kconv(A, dv, Q[w], qd[w], C[w], dv);
                free(pws);
            } else if (variant == MVDO_OPT1) {
                mvdo_kconv(A, dv, Pn[w], dw, C[w], dv);
            } else {
                for (long i = 0; i < Tv; ++i) C[w][i] = A[i];
            }
            for (long i = 0; i < Tv; ++i) U[i] *= C[w][i];
        }
    }
    double su = 0.0, kk = 0.0;
    for (long i = 0; i < Tv; ++i) su += U[i];
    for (long i = 0; i < Tv; ++i) kk += Kb[i] * (U[i] / su);
    double* Ub = (double*)malloc(sizeof(double) * Tv);
    for (long i = 0; i < Tv; ++i) Ub[i] = (Kb[i] - kk) / su; /* through K = U / sum(U) */
    double* Ab = (double*)calloc(Tv, sizeof(double));
    for (long i = 0; i < Tv; ++i) {
        double prod = 1.0;
        for (int w = 0; w < nv; ++w)
            if (C[w]) prod *= C[w][i];
        Ab[i] += Ub[i] * prod; /* U = A . prod C_w */
    }
    for (int w = 0; w < nv; ++w) {
        if (!C[w]) continue;
        const int* dw = pd + 3 * w;
        double* Cb = (double*)malloc(sizeof(double) * Tv);
        for (long i = 0; i < Tv; ++i) {
            double prod = A[i];
            for (int u = 0; u < nv; ++u)
                if (C[u] && u != w) prod *= C[u][i];
            Cb[i] = Ub[i] * prod;
        }
        if (variant == MVDO_OPT2) { /* C_w = A */
            for (long i = 0; i < Tv; ++i) Ab[i] += Cb[i];
        } else {
            /* C_w(d) = sum_e A(e) G(d - e), G = Q_w (Eq. 222) or P_w (Eq. 230) */
            const double* G = variant == MVDO_EFFICIENT ? Q[w] : Pn[w];
            const int* gd = variant == MVDO_EFFICIENT ? qd[w] : dw;
            const int ghx = (gd[0] - 1) / 2, ghy = (gd[1] - 1) / 2, ghz = (gd[2] - 1) / 2;
            const long Tg = (long)gd[0] * gd[1] * gd[2];
            double* Gb = (double*)calloc(Tg, sizeof(double));
            for (long ie = 0; ie < Tv; ++ie) {
                const int ex = (int)(ie % dv[0]) - hvx, ey = (int)((ie / dv[0]) % dv[1]) - hvy,
                          ez = (int)(ie / ((long)dv[0] * dv[1])) - hvz;
                for (long id = 0; id < Tv; ++id) {
                    const int dx = (int)(id % dv[0]) - hvx, dy = (int)((id / dv[0]) % dv[1]) - hvy,
                              dz = (int)(id / ((long)dv[0] * dv[1])) - hvz;
                    const int fx = dx - ex, fy = dy - ey, fz = dz - ez;
                    if (fx < -ghx || fx > ghx || fy < -ghy || fy > ghy || fz < -ghz || fz > ghz) continue;
                    const long ig = idx3(fx + ghx, fy + ghy, fz + ghz, gd[0], gd[1]);
                    Ab[ie] += Cb[id] * G[ig];
                    Gb[ig] += Cb[id] * A[ie];
                }
            }
            if (variant == MVDO_EFFICIENT) {
                /* Q_w(f) = sum_g Pn_w(g) Pn_w(g - f): dQ(f)/dPn_w(h) = Pn_w(h - f) + Pn_w(h + f) */
                const int hwx = (dw[0] - 1) / 2, hwy = (dw[1] - 1) / 2, hwz = (dw[2] - 1) / 2;
                const long Tw = (long)dw[0] * dw[1] * dw[2];
                for (long ih = 0; ih < Tw; ++ih) {
                    const int hx = (int)(ih % dw[0]) - hwx, hy = (int)((ih / dw[0]) % dw[1]) - hwy,
                              hz = (int)(ih / ((long)dw[0] * dw[1])) - hwz;
                    double s = 0.0;
                    for (long ig = 0; ig < Tg; ++ig) {
                        const int fx = (int)(ig % gd[0]) - ghx, fy = (int)((ig / gd[0]) % gd[1]) - ghy,
                                  fz = (int)(ig / ((long)gd[0] * gd[1])) - ghz;
                        s += Gb[ig] * (kat(Pn[w], dw, hx - fx, hy - fy, hz - fz) + kat(Pn[w], dw, hx + fx, hy + fy, hz + fz));
                    }
                    Pb[w][ih] += s;
                }
            } else {
                const long Tw = (long)dw[0] * dw[1] * dw[2];
                for (long i = 0; i < Tw; ++i) Pb[w][i] += Gb[i];
            }
            free(Gb);
        }
        free(Cb);
    }
    /* A = Pn_v^*: Pn_v(d) = A(-d) */
    for (long i = 0; i < Tv; ++i) {
        const int x = (int)(i % dv[0]), y = (int)((i / dv[0]) % dv[1]), z = (int)(i / ((long)dv[0] * dv[1]));
        Pb[v][idx3(dv[0] - 1 - x, dv[1] - 1 - y, dv[2] - 1 - z, dv[0], dv[1])] += Ab[i];
    }
    for (int w = 0; w < nv; ++w) {
        free(C[w]);
        free(Q[w]);
    }
    free(C);
    free(Q);
    free(qd);
    free(A);
    free(U);
    free(Ub);
    free(Ab);
}

/* Loss and gradients of the unrolled iteration (see the block comment).
 * grad_views: nv volumes; grad_psfs: nv boxes of the RAW PSFs as given.
 * Returns the loss, or -1 on error. psiK (optional) receives the estimate. */
double mvdo_unrolled_grad(int nv, const double* const* views, const double* const* psfs, const int* pd,
                          const int dims[3], int variant, int n_iter, const double* truth, double* const* grad_views,
                          double* const* grad_psfs, double* psiK) {
    const long M = (long)dims[0] * dims[1] * dims[2];
    double** Pn = (double**)malloc(sizeof(double*) * nv);
    double** K = (double**)malloc(sizeof(double*) * nv);
    double** Pb = (double**)malloc(sizeof(double*) * nv);
    double** Kb = (double**)malloc(sizeof(double*) * nv);
    double* psum = (double*)malloc(sizeof(double) * nv);
    for (int v = 0; v < nv; ++v) {
        const long T = (long)pd[3 * v] * pd[3 * v + 1] * pd[3 * v + 2];
        double s = 0.0;
        for (long i = 0; i < T; ++i) s += psfs[v][i];
        psum[v] = s;
        Pn[v] = (double*)malloc(sizeof(double) * T);
        for (long i = 0; i < T; ++i) Pn[v][i] = psfs[v][i] / s;
        Pb[v] = (double*)calloc(T, sizeof(double));
        Kb[v] = (double*)calloc(T, sizeof(double));
    }
    for (int v = 0; v < nv; ++v) {
        const long T = (long)pd[3 * v] * pd[3 * v + 1] * pd[3 * v + 2];
        K[v] = (double*)malloc(sizeof(double) * T);
        mvdo_compound(nv, (const double* const*)Pn, pd, v, variant, K[v]);
    }
    const double psi0 = mvdo_mean_views(nv, views, dims);
    const double eps = 1e-4 * psi0;
    const long nup = (long)n_iter * nv;
    double* hist = (double*)malloc(sizeof(double) * M * (nup + 1));
    for (long i = 0; i < M; ++i) hist[i] = psi0;
    double *b = (double*)malloc(sizeof(double) * M), *r = (double*)malloc(sizeof(double) * M),
           *c = (double*)malloc(sizeof(double) * M);
    for (long u = 0; u < nup; ++u) {
        const int v = (int)(u % nv);
        for (long i = 0; i < M; ++i) hist[(u + 1) * M + i] = hist[u * M + i];
        mvdo_update(hist + (u + 1) * M, views[v], Pn[v], pd + 3 * v, K[v], pd + 3 * v, dims, eps, b, r, c);
    }
    const double* pk = hist + nup * M;
    double loss = 0.0;
    double* g = (double*)malloc(sizeof(double) * M);
    for (long i = 0; i < M; ++i) {
        const double d = pk[i] - truth[i];
        loss += d * d;
        g[i] = 2.0 * d / (double)M;
    }
    loss /= (double)M;
    if (psiK)
        for (long i = 0; i < M; ++i) psiK[i] = pk[i];
    for (int v = 0; v < nv; ++v)
        for (long i = 0; i < M; ++i) grad_views[v][i] = 0.0;
    double *cb = (double*)malloc(sizeof(double) * M), *rb = (double*)malloc(sizeof(double) * M),
           *bb = (double*)malloc(sizeof(double) * M), *tmp = (double*)malloc(sizeof(double) * M);
    for (long u = nup - 1; u >= 0; --u) {
        const int v = (int)(u % nv);
        const int* kd = pd + 3 * v;
        const long T = (long)kd[0] * kd[1] * kd[2];
        const double* psi = hist + u * M;
        /* recompute the forward intermediates of this update */
        mvdo_conv(psi, dims, Pn[v], kd, b);
        for (long i = 0; i < M; ++i) r[i] = views[v][i] / fmax(b[i], eps);
        mvdo_conv(r, dims, K[v], kd, c);
        double* gnew = tmp;
        for (long i = 0; i < M; ++i) {
            const double t = psi[i] * c[i];
            const double tb = t > eps ? g[i] : 0.0;
            gnew[i] = tb * c[i];
            cb[i] = tb * psi[i];
        }
        double* Ks = (double*)malloc(sizeof(double) * T);
        double* kg = (double*)malloc(sizeof(double) * T);
        mvdo_mirror(K[v], kd, Ks);
        mvdo_conv(cb, dims, Ks, kd, rb);
        corr_box(cb, r, dims, kd, kg);
        for (long i = 0; i < T; ++i) Kb[v][i] += kg[i];
        for (long i = 0; i < M; ++i) {
            const double bp = fmax(b[i], eps);
            grad_views[v][i] += rb[i] / bp;
            bb[i] = b[i] > eps ? -rb[i] * r[i] / bp : 0.0;
        }
        double* Ps = Ks;
        mvdo_mirror(Pn[v], kd, Ps);
        mvdo_conv(bb, dims, Ps, kd, c);
        for (long i = 0; i < M; ++i) gnew[i] += c[i];
        corr_box(bb, psi, dims, kd, kg);
        for (long i = 0; i < T; ++i) Pb[v][i] += kg[i];
        free(Ks);
        free(kg);
        double* sw = g;
        g = gnew;
        tmp = sw;
    }
    /* flat start psi0 = mean of all views */
    double gs = 0.0;
    for (long i = 0; i < M; ++i) gs += g[i];
    for (int v = 0; v < nv; ++v)
        for (long i = 0; i < M; ++i) grad_views[v][i] += gs / ((double)M * nv);
    for (int v = 0; v < nv; ++v) compound_vjp(nv, Pn, pd, v, variant, Kb[v], Pb);
    /* PSF normalisation Pn = p / sum(p) */
    for (int v = 0; v < nv; ++v) {
        const long T = (long)pd[3 * v] * pd[3 * v + 1] * pd[3 * v + 2];
        double dot = 0.0;
        for (long i = 0; i < T; ++i) dot += Pb[v][i] * Pn[v][i];
        for (long i = 0; i < T; ++i) grad_psfs[v][i] = (Pb[v][i] - dot) / psum[v];
    }
    for (int v = 0; v < nv; ++v) {
        free(Pn[v]);
        free(K[v]);
        free(Pb[v]);
        free(Kb[v]);
    }
    free(Pn);
    free(K);
    free(Pb);
    free(Kb);
    free(psum);
    free(hist);
    free(b);
    free(r);
    free(c);
    free(g);
    free(cb);
    free(rb);
    free(bb);
    free(tmp);
    return loss;
}
