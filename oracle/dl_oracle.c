/*
 * FP64 CPU oracle for dictionary learning with Jacobi atom updates
 * (Irofti & Dumitrescu, "Overcomplete Dictionary Learning with Jacobi Atom
 * Updates", arXiv 1509.05054).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * statement of what the GPU library computes.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or helper with the CUDA library, and the CUDA library never
 * calls it.
 *
 * Conventions (all arrays are plain host memory, double precision):
 *   Y  p x m, column-major: signal i is Y[i*p .. i*p+p)            (Eq. 1)
 *   D  p x n, column-major: atom j is D[j*p .. j*p+p)               (Eq. 1)
 *   X  n x m with at most s nonzeros per column, stored per signal in
 *      "slots": idx[i*s + t], val[i*s + t] for t < cnt[i], atoms ascending.
 *
 * Readings of points the paper leaves open (each also listed in the design
 * notes of the repository):
 *   - OMP argmax ties go to the lowest atom index; selected atoms are masked
 *     explicitly.
 *   - OMP stops early when max|alpha| = 0, when the new Cholesky pivot
 *     delta <= 1e-12 (dependent atom), or when the residual energy falls to
 *     1e-14 ||y||^2.  Fewer than s nonzeros is allowed by "at most s" (Eq. 1).
 *   - An atom no signal uses (I_j empty), or whose power-iteration vector
 *     F x^T is exactly zero, is left unchanged.
 *
 * Parity pins: every function here is checked by tests/test_oracle_pins.py
 * against brute force, closed forms, invariants and Table 1 of the paper.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_DELTA_MIN 1e-12
#define ORACLE_RESID_REL 1e-14

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* G = D^T D, the Gram matrix Batch-OMP works from ([RZE08], cited for the
 * OMP-Box tool in Section 4). G is n x n, G[a*n + b] = d_a . d_b. */
void oracle_gram(int p, int n, const double* D, double* G, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel for schedule(static)
    for (int a = 0; a < n; ++a) {
        for (int b = 0; b < n; ++b) {
            double acc = 0.0;
            for (int r = 0; r < p; ++r) acc += D[(size_t)a * p + r] * D[(size_t)b * p + r];
            G[(size_t)a * n + b] = acc;
        }
    }
}

/* Sort the first k (atom, value) pairs by ascending atom index (insertion sort). */
static void sort_pairs(int k, int32_t* idx, double* val) {
    for (int a = 1; a < k; ++a) {
        int32_t ti = idx[a];
        double tv = val[a];
        int b = a - 1;
        while (b >= 0 && idx[b] > ti) {
            idx[b + 1] = idx[b];
            val[b + 1] = val[b];
            --b;
        }
        idx[b + 1] = ti;
        val[b + 1] = tv;
    }
}

/*
 * Batch-OMP for one signal (OMP of Section 1 / Algorithm 1 step 1, in the
 * Cholesky form of the OMP-Box tool named in Section 4):
 *   alpha0 = D^T y, alpha = alpha0, I = {}
 *   for k = 1..s:
 *     idx = argmax_{j not in I} |alpha_j|            (stop if the max is 0)
 *     w = L^{-1} G[I, idx];  delta = G[idx,idx] - w.w (stop if delta <= 1e-12)
 *     L <- [[L, 0], [w^T, sqrt(delta)]];  I <- I + {idx}
 *     solve L L^T gamma = alpha0_I
 *     alpha = alpha0 - G[:, I] gamma
 *     stop if ||y - D_I gamma||^2 = ||y||^2 - gamma.alpha0_I <= 1e-14 ||y||^2
 * Returns the number of selected atoms; idx/val hold the support (ascending)
 * and the coefficients gamma.
 * `gap` (may be NULL) receives, per step, the relative gap between the
 * largest and second-largest unselected |alpha| -- used by tests to decide
 * whether a support mismatch is a legitimate near-tie.
 */
static int omp_batch_one(int n, int s, const double* G, const double* a0, double yy,
                         double* alpha, double* L, double* w, double* z, double* gamma,
                         unsigned char* sel, int32_t* I, int32_t* idx_out, double* val_out,
                         double* gap) {
    memcpy(alpha, a0, sizeof(double) * (size_t)n);
    memset(sel, 0, (size_t)n);
    int k = 0;
    while (k < s) {
        int best = -1, second_set = 0;
        double bv = 0.0, sv = 0.0;
        for (int j = 0; j < n; ++j) {
            if (sel[j]) continue;
            double v = fabs(alpha[j]);
            if (best < 0 || v > bv) {
                if (best >= 0) { sv = bv; second_set = 1; }
                bv = v;
                best = j;
            } else if (!second_set || v > sv) {
                sv = v;
                second_set = 1;
            }
        }
        if (gap) gap[k] = (best >= 0 && bv > 0.0 && second_set) ? (bv - sv) / bv : 1.0;
        if (best < 0 || bv <= 0.0) break;
        /* Cholesky row append: L w = G[I, idx] */
        double delta = G[(size_t)best * n + best];
        for (int a = 0; a < k; ++a) {
            double acc = G[(size_t)I[a] * n + best];
            for (int b = 0; b < a; ++b) acc -= L[a * s + b] * w[b];
            w[a] = acc / L[a * s + a];
            delta -= w[a] * w[a];
        }
        if (delta <= ORACLE_DELTA_MIN) break;
        for (int b = 0; b < k; ++b) L[k * s + b] = w[b];
        L[k * s + k] = sqrt(delta);
        I[k] = best;
        sel[best] = 1;
        ++k;
        /* L z = alpha0_I, then L^T gamma = z */
        for (int a = 0; a < k; ++a) {
            double acc = a0[I[a]];
            for (int b = 0; b < a; ++b) acc -= L[a * s + b] * z[b];
            z[a] = acc / L[a * s + a];
        }
        for (int a = k - 1; a >= 0; --a) {
            double acc = z[a];
            for (int b = a + 1; b < k; ++b) acc -= L[b * s + a] * gamma[b];
            gamma[a] = acc / L[a * s + a];
        }
        /* alpha = alpha0 - G[:, I] gamma */
        for (int j = 0; j < n; ++j) {
            double acc = a0[j];
            for (int a = 0; a < k; ++a) acc -= G[(size_t)j * n + I[a]] * gamma[a];
            alpha[j] = acc;
        }
        double rr = yy;
        for (int a = 0; a < k; ++a) rr -= gamma[a] * a0[I[a]];
        if (rr <= ORACLE_RESID_REL * yy) break;
    }
    for (int a = 0; a < k; ++a) {
        idx_out[a] = I[a];
        val_out[a] = gamma[a];
    }
    sort_pairs(k, idx_out, val_out);
    return k;
}

/*
 * Batch-OMP over all m signals. idx/val are m*s slots, cnt is m counts.
 * gaps (may be NULL) is m*s: per signal and step, the relative top-two gap.
 * Returns 0.
 */
int oracle_omp(int p, int n, int64_t m, const double* Y, const double* D, int s,
               int32_t* idx, double* val, int32_t* cnt, double* gaps, int nthreads) {
    set_threads(nthreads);
    double* G = (double*)malloc(sizeof(double) * (size_t)n * n);
    oracle_gram(p, n, D, G, nthreads);
#pragma omp parallel
    {
        double* a0 = (double*)malloc(sizeof(double) * (size_t)n);
        double* alpha = (double*)malloc(sizeof(double) * (size_t)n);
        double* L = (double*)calloc((size_t)s * s, sizeof(double));
        double* w = (double*)malloc(sizeof(double) * (size_t)s);
        double* z = (double*)malloc(sizeof(double) * (size_t)s);
        double* gamma = (double*)malloc(sizeof(double) * (size_t)s);
        unsigned char* sel = (unsigned char*)malloc((size_t)n);
        int32_t* I = (int32_t*)malloc(sizeof(int32_t) * (size_t)s);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < m; ++i) {
            const double* y = Y + (size_t)i * p;
            double yy = 0.0;
            for (int r = 0; r < p; ++r) yy += y[r] * y[r];
            for (int j = 0; j < n; ++j) {
                double acc = 0.0;
                for (int r = 0; r < p; ++r) acc += D[(size_t)j * p + r] * y[r];
                a0[j] = acc;
            }
            int k = omp_batch_one(n, s, G, a0, yy, alpha, L, w, z, gamma, sel, I,
                                  idx + (size_t)i * s, val + (size_t)i * s,
                                  gaps ? gaps + (size_t)i * s : NULL);
            for (int t = k; t < s; ++t) {
                idx[(size_t)i * s + t] = -1;
                val[(size_t)i * s + t] = 0.0;
                if (gaps) gaps[(size_t)i * s + t] = 1.0;
            }
            cnt[i] = k;
        }
        free(a0); free(alpha); free(L); free(w); free(z); free(gamma); free(sel); free(I);
    }
    free(G);
    return 0;
}

/*
 * Solve the k x k system A x = b in place by Gaussian elimination with
 * partial pivoting (A row-major, destroyed). Returns the smallest absolute
 * pivot met.
 */
static double gauss_solve(int k, double* A, double* b) {
    double minpiv = INFINITY;
    for (int c = 0; c < k; ++c) {
        int pr = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(A[r * k + c]) > fabs(A[pr * k + c])) pr = r;
        if (pr != c) {
            for (int q = 0; q < k; ++q) {
                double t = A[c * k + q]; A[c * k + q] = A[pr * k + q]; A[pr * k + q] = t;
            }
            double t = b[c]; b[c] = b[pr]; b[pr] = t;
        }
        double piv = A[c * k + c];
        if (fabs(piv) < minpiv) minpiv = fabs(piv);
        if (piv == 0.0) return 0.0;
        for (int r = c + 1; r < k; ++r) {
            double f = A[r * k + c] / piv;
            for (int q = c; q < k; ++q) A[r * k + q] -= f * A[c * k + q];
            b[r] -= f * b[c];
        }
    }
    for (int c = k - 1; c >= 0; --c) {
        double acc = b[c];
        for (int q = c + 1; q < k; ++q) acc -= A[c * k + q] * b[q];
        b[c] = acc / A[c * k + c];
    }
    return minpiv;
}

/*
 * Textbook OMP (Pati et al., cited in Section 1) written independently of the
 * Batch-OMP form above: the residual r is kept explicitly, correlations are
 * D^T r, and the coefficients come from a fresh solve of the normal equations
 * (D_I^T D_I) gamma = D_I^T y each step. Same tie and stop rules; the
 * dependent-atom test uses the energy of the new atom's component orthogonal
 * to span(D_I), ||d||^2 - d^T D_I (D_I^T D_I)^{-1} D_I^T d.
 */
int oracle_omp_naive(int p, int n, int64_t m, const double* Y, const double* D, int s,
                     int32_t* idx, double* val, int32_t* cnt, int nthreads) {
    set_threads(nthreads);
#pragma omp parallel
    {
        double* r = (double*)malloc(sizeof(double) * (size_t)p);
        double* c = (double*)malloc(sizeof(double) * (size_t)n);
        double* A = (double*)malloc(sizeof(double) * (size_t)s * s);
        double* b = (double*)malloc(sizeof(double) * (size_t)s);
        double* gam = (double*)malloc(sizeof(double) * (size_t)s);
        unsigned char* sel = (unsigned char*)malloc((size_t)n);
        int32_t* I = (int32_t*)malloc(sizeof(int32_t) * (size_t)s);
#pragma omp for schedule(dynamic, 64)
        for (int64_t i = 0; i < m; ++i) {
            const double* y = Y + (size_t)i * p;
            double yy = 0.0;
            for (int q = 0; q < p; ++q) { r[q] = y[q]; yy += y[q] * y[q]; }
            memset(sel, 0, (size_t)n);
            int k = 0;
            while (k < s) {
                for (int j = 0; j < n; ++j) {
                    double acc = 0.0;
                    for (int q = 0; q < p; ++q) acc += D[(size_t)j * p + q] * r[q];
                    c[j] = acc;
                }
                int best = -1;
                double bv = 0.0;
                for (int j = 0; j < n; ++j) {
                    if (sel[j]) continue;
                    if (best < 0 || fabs(c[j]) > bv) { bv = fabs(c[j]); best = j; }
                }
                if (best < 0 || bv <= 0.0) break;
                if (k > 0) {
                    /* dependent-atom energy of the candidate */
                    const double* dn = D + (size_t)best * p;
                    for (int a = 0; a < k; ++a) {
                        for (int q2 = 0; q2 < k; ++q2) {
                            double acc = 0.0;
                            for (int q = 0; q < p; ++q)
                                acc += D[(size_t)I[a] * p + q] * D[(size_t)I[q2] * p + q];
                            A[a * k + q2] = acc;
                        }
                        double acc = 0.0;
                        for (int q = 0; q < p; ++q) acc += D[(size_t)I[a] * p + q] * dn[q];
                        b[a] = acc;
                        gam[a] = acc;
                    }
                    gauss_solve(k, A, b);
                    double e = 0.0;
                    for (int q = 0; q < p; ++q) e += dn[q] * dn[q];
                    for (int a = 0; a < k; ++a) e -= gam[a] * b[a];
                    if (e <= ORACLE_DELTA_MIN) break;
                }
                I[k] = best;
                sel[best] = 1;
                ++k;
                for (int a = 0; a < k; ++a) {
                    for (int q2 = 0; q2 < k; ++q2) {
                        double acc = 0.0;
                        for (int q = 0; q < p; ++q)
                            acc += D[(size_t)I[a] * p + q] * D[(size_t)I[q2] * p + q];
                        A[a * k + q2] = acc;
                    }
                    double acc = 0.0;
                    for (int q = 0; q < p; ++q) acc += D[(size_t)I[a] * p + q] * y[q];
                    b[a] = acc;
                }
                gauss_solve(k, A, b);
                for (int a = 0; a < k; ++a) gam[a] = b[a];
                double rr = 0.0;
                for (int q = 0; q < p; ++q) {
                    double acc = y[q];
                    for (int a = 0; a < k; ++a) acc -= D[(size_t)I[a] * p + q] * gam[a];
                    r[q] = acc;
                    rr += acc * acc;
                }
                if (rr <= ORACLE_RESID_REL * yy) break;
            }
            for (int a = 0; a < k; ++a) {
                idx[(size_t)i * s + a] = I[a];
                val[(size_t)i * s + a] = gam[a];
            }
            sort_pairs(k, idx + (size_t)i * s, val + (size_t)i * s);
            for (int t = k; t < s; ++t) {
                idx[(size_t)i * s + t] = -1;
                val[(size_t)i * s + t] = 0.0;
            }
            cnt[i] = k;
        }
        free(r); free(c); free(A); free(b); free(gam); free(sel); free(I);
    }
    return 0;
}

/* E = Y - D X for all signals (Eq. 1). E is p x m column-major. */
static void form_error(int p, int64_t m, const double* Y, const double* D, int s,
                       const int32_t* idx, const double* val, const int32_t* cnt, double* E) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double* e = E + (size_t)i * p;
        const double* y = Y + (size_t)i * p;
        for (int q = 0; q < p; ++q) e[q] = y[q];
        for (int t = 0; t < cnt[i]; ++t) {
            const double* d = D + (size_t)idx[(size_t)i * s + t] * p;
            double x = val[(size_t)i * s + t];
            for (int q = 0; q < p; ++q) e[q] -= d[q] * x;
        }
    }
}

/* ||Y - D X||_F^2 and ||Y||_F^2 (the relative RMSE of Section 4.2 is the
 * square root of their ratio). */
void oracle_error_energy(int p, int64_t m, const double* Y, const double* D, int s,
                         const int32_t* idx, const double* val, const int32_t* cnt,
                         double* out2, int nthreads) {
    set_threads(nthreads);
    double ee = 0.0, yy = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ee, yy)
    for (int64_t i = 0; i < m; ++i) {
        const double* y = Y + (size_t)i * p;
        for (int q = 0; q < p; ++q) {
            double acc = y[q];
            for (int t = 0; t < cnt[i]; ++t)
                acc -= D[(size_t)idx[(size_t)i * s + t] * p + q] * val[(size_t)i * s + t];
            ee += acc * acc;
            yy += y[q] * y[q];
        }
    }
    out2[0] = ee;
    out2[1] = yy;
}

/* Index sets I_j (Section 3): for every atom j, the slots (i*s + t) of the
 * signals whose representation uses atom j, in ascending signal order. */
static void build_index_sets(int n, int64_t m, int s, const int32_t* idx, const int32_t* cnt,
                             int64_t* start, int64_t* slots) {
    for (int j = 0; j <= n; ++j) start[j] = 0;
    for (int64_t i = 0; i < m; ++i)
        for (int t = 0; t < cnt[i]; ++t) start[idx[(size_t)i * s + t] + 1]++;
    for (int j = 0; j < n; ++j) start[j + 1] += start[j];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    for (int j = 0; j < n; ++j) fill[j] = start[j];
    for (int64_t i = 0; i < m; ++i)
        for (int t = 0; t < cnt[i]; ++t) {
            int j = idx[(size_t)i * s + t];
            slots[fill[j]++] = (int64_t)i * s + t;
        }
    free(fill);
}

enum { ORACLE_RULE_AKSVD = 0, ORACLE_RULE_SGK = 1, ORACLE_RULE_NSGK = 2 };

/*
 * Atom-update stage with group size ntilde (Algorithm 1 steps 2-5, with the
 * P-SGK structure of Algorithm 2): for every group of ntilde consecutive
 * atoms, E = Y - D X is formed from the current D and X; then for each atom j
 * of the group, independently,
 *     F = E_{I_j} + d_j x_{j,I_j}                                   (Eq. 3)
 *   AK-SVD (rule 0):  d_j = F x^T / ||F x^T||,  x_{j,I_j} = F^T d_j   (Eq. 5)
 *   SGK    (rule 1):  d_j = F x^T / (x x^T),  then d_j /= ||d_j||   (Eq. 6)
 * ntilde = n is the fully parallel (Jacobi) form PAK-SVD / P-SGK;
 * ntilde = 1 is the sequential Gauss-Seidel form (Eq. 2).
 * only_atom >= 0 restricts the update to that one atom (the others are left
 * as they are); -1 updates all atoms.
 * D (p x n) and val (m*s slots) are updated in place; the support is fixed.
 * unused (may be NULL) receives the number of atoms left unchanged because
 * I_j was empty or F x^T was zero.
 */
int oracle_atom_update(int p, int n, int64_t m, const double* Y, double* D, int s,
                       const int32_t* idx, double* val, const int32_t* cnt, int ntilde,
                       int rule, int only_atom, int* unused, int nthreads) {
    set_threads(nthreads);
    if (ntilde < 1) ntilde = 1;
    double* E = (double*)malloc(sizeof(double) * (size_t)p * m);
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* slots = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m * s + 1));
    double* Dnew = (double*)malloc(sizeof(double) * (size_t)p * n);
    double* vnew = (double*)malloc(sizeof(double) * (size_t)(m * s + 1));
    build_index_sets(n, m, s, idx, cnt, start, slots);
    int n_unused = 0;
    for (int g0 = 0; g0 < n; g0 += ntilde) {
        int g1 = g0 + ntilde < n ? g0 + ntilde : n;
        form_error(p, m, Y, D, s, idx, val, cnt, E);
        memcpy(Dnew, D, sizeof(double) * (size_t)p * n);
        memcpy(vnew, val, sizeof(double) * (size_t)(m * s));
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_unused)
        for (int j = g0; j < g1; ++j) {
            if (only_atom >= 0 && j != only_atom) continue;
            int64_t nI = start[j + 1] - start[j];
            if (nI == 0) { n_unused++; continue; }
            const double* dj = D + (size_t)j * p;
            /* F = E_I + d_j x_{j,I}, explicit p x |I| matrix, column c <-> slot */
            double* F = (double*)malloc(sizeof(double) * (size_t)p * nI);
            double* x = (double*)malloc(sizeof(double) * (size_t)nI);
            for (int64_t c = 0; c < nI; ++c) {
                int64_t sl = slots[start[j] + c];
                int64_t i = sl / s;
                x[c] = val[sl];
                for (int q = 0; q < p; ++q)
                    F[(size_t)c * p + q] = E[(size_t)i * p + q] + dj[q] * x[c];
            }
            double* g = (double*)calloc((size_t)p, sizeof(double));
            for (int64_t c = 0; c < nI; ++c)
                for (int q = 0; q < p; ++q) g[q] += F[(size_t)c * p + q] * x[c];
            double gn = 0.0;
            for (int q = 0; q < p; ++q) gn += g[q] * g[q];
            if (rule == ORACLE_RULE_SGK) {
                double xx = 0.0;
                for (int64_t c = 0; c < nI; ++c) xx += x[c] * x[c];
                if (xx > 0.0) for (int q = 0; q < p; ++q) g[q] /= xx;
                gn = 0.0;
                for (int q = 0; q < p; ++q) gn += g[q] * g[q];
            }
            double* dn = Dnew + (size_t)j * p;
            if (gn > 0.0) {
                double inv = 1.0 / sqrt(gn);
                for (int q = 0; q < p; ++q) dn[q] = g[q] * inv;
            } else {
                n_unused++;
                for (int q = 0; q < p; ++q) dn[q] = dj[q];
            }
            if (rule == ORACLE_RULE_AKSVD) {
                for (int64_t c = 0; c < nI; ++c) {
                    double acc = 0.0;
                    for (int q = 0; q < p; ++q) acc += F[(size_t)c * p + q] * dn[q];
                    vnew[slots[start[j] + c]] = acc;
                }
            }
            free(F); free(x); free(g);
        }
        memcpy(D, Dnew, sizeof(double) * (size_t)p * n);
        memcpy(val, vnew, sizeof(double) * (size_t)(m * s));
    }
    if (unused) *unused = n_unused;
    free(E); free(start); free(slots); free(Dnew); free(vnew);
    return 0;
}

/*
 * P-NSGK atom-update stage (Section 3, Eq. 7): SGK with the signal matrix Y
 * replaced by Z = Y + D X_prev - D X, where D is the dictionary the iteration
 * started from, X the representations its sparse coding produced and X_prev
 * those at the beginning of the iteration; the representations entering the
 * SGK update are X_prev's (supports and values).  For every group of ntilde
 * consecutive atoms, E = Z - D X_prev with the current D; then for each atom j
 * of the group, independently, with I_j the signals whose X_prev column uses j,
 *     F = E_{I_j} + d_j xp_{j,I_j},   d_j = F xp^T / (xp xp^T),  d_j /= ||d_j||
 * (atoms with an empty I_j, or F xp^T = 0, are left unchanged and counted).
 * Neither X nor X_prev is modified.  With X_prev = X this is the SGK rule of
 * oracle_atom_update.
 */
int oracle_atom_update_nsgk(int p, int n, int64_t m, const double* Y, double* D, int s,
                            const int32_t* idx, const double* val, const int32_t* cnt,
                            const int32_t* pidx, const double* pval, const int32_t* pcnt,
                            int ntilde, int* unused, int nthreads) {
    set_threads(nthreads);
    if (ntilde < 1) ntilde = 1;
    double* Z = (double*)malloc(sizeof(double) * (size_t)p * m);
    double* E = (double*)malloc(sizeof(double) * (size_t)p * m);
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t* slots = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m * s + 1));
    double* Dnew = (double*)malloc(sizeof(double) * (size_t)p * n);
    /* Z = (Y - D X) + D X_prev, with the entry dictionary */
    form_error(p, m, Y, D, s, idx, val, cnt, Z);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        double* z = Z + (size_t)i * p;
        for (int u = 0; u < pcnt[i]; ++u) {
            const double* d = D + (size_t)pidx[(size_t)i * s + u] * p;
            double x = pval[(size_t)i * s + u];
            for (int q = 0; q < p; ++q) z[q] += d[q] * x;
        }
    }
    build_index_sets(n, m, s, pidx, pcnt, start, slots);
    int n_unused = 0;
    for (int g0 = 0; g0 < n; g0 += ntilde) {
        int g1 = g0 + ntilde < n ? g0 + ntilde : n;
        form_error(p, m, Z, D, s, pidx, pval, pcnt, E);   /* E = Z - D X_prev */
        memcpy(Dnew, D, sizeof(double) * (size_t)p * n);
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : n_unused)
        for (int j = g0; j < g1; ++j) {
            int64_t nI = start[j + 1] - start[j];
            if (nI == 0) { n_unused++; continue; }
            const double* dj = D + (size_t)j * p;
            double* g = (double*)calloc((size_t)p, sizeof(double));
            double xx = 0.0;
            for (int64_t c = 0; c < nI; ++c) {
                int64_t sl = slots[start[j] + c];
                int64_t i = sl / s;
                double x = pval[sl];
                xx += x * x;
                for (int q = 0; q < p; ++q) g[q] += (E[(size_t)i * p + q] + dj[q] * x) * x;
            }
            double gn = 0.0;
            if (xx > 0.0) for (int q = 0; q < p; ++q) g[q] /= xx;
            for (int q = 0; q < p; ++q) gn += g[q] * g[q];
            double* dn = Dnew + (size_t)j * p;
            if (gn > 0.0) {
                double inv = 1.0 / sqrt(gn);
                for (int q = 0; q < p; ++q) dn[q] = g[q] * inv;
            } else {
                n_unused++;
                for (int q = 0; q < p; ++q) dn[q] = dj[q];
            }
            free(g);
        }
        memcpy(D, Dnew, sizeof(double) * (size_t)p * n);
    }
    if (unused) *unused = n_unused;
    free(Z); free(E); free(start); free(slots); free(Dnew);
    return 0;
}

/*
 * The DL iteration of Algorithm 1, repeated `iters` times: OMP with the
 * current D (step 1), then the atom-update stage with group size ntilde and
 * the chosen rule (AK-SVD, SGK, or P-NSGK with the representations of the
 * previous iteration; the first iteration, having none, uses its own and so is
 * P-SGK). rmse[2*k] is ||Y - D^(k) X^(k)||_F / ||Y||_F right after
 * sparse coding, rmse[2*k+1] the same with the updated D and (for AK-SVD)
 * updated X at the end of the iteration (Section 4.2 computes the errors at
 * the end of an iteration). On return idx/val/cnt hold the last X.
 */
int oracle_dl(int p, int n, int64_t m, const double* Y, double* D, int s, int iters,
              int ntilde, int rule, int32_t* idx, double* val, int32_t* cnt, double* rmse,
              int nthreads) {
    double e2[2];
    /* P-NSGK keeps the representations the iteration started from; the first
       iteration has none and uses its own (it is then P-SGK) */
    int32_t* pidx = NULL;
    double* pval = NULL;
    int32_t* pcnt = NULL;
    if (rule == ORACLE_RULE_NSGK) {
        pidx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m * s + 1));
        pval = (double*)malloc(sizeof(double) * (size_t)(m * s + 1));
        pcnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    }
    for (int it = 0; it < iters; ++it) {
        oracle_omp(p, n, m, Y, D, s, idx, val, cnt, NULL, nthreads);
        oracle_error_energy(p, m, Y, D, s, idx, val, cnt, e2, nthreads);
        if (rmse) rmse[2 * it] = e2[1] > 0 ? sqrt(e2[0] / e2[1]) : 0.0;
        if (rule == ORACLE_RULE_NSGK) {
            if (it == 0) {
                memcpy(pidx, idx, sizeof(int32_t) * (size_t)(m * s));
                memcpy(pval, val, sizeof(double) * (size_t)(m * s));
                memcpy(pcnt, cnt, sizeof(int32_t) * (size_t)m);
            }
            oracle_atom_update_nsgk(p, n, m, Y, D, s, idx, val, cnt, pidx, pval, pcnt, ntilde,
                                    NULL, nthreads);
            memcpy(pidx, idx, sizeof(int32_t) * (size_t)(m * s));
            memcpy(pval, val, sizeof(double) * (size_t)(m * s));
            memcpy(pcnt, cnt, sizeof(int32_t) * (size_t)m);
        } else {
            oracle_atom_update(p, n, m, Y, D, s, idx, val, cnt, ntilde, rule, -1, NULL, nthreads);
        }
        oracle_error_energy(p, m, Y, D, s, idx, val, cnt, e2, nthreads);
        if (rmse) rmse[2 * it + 1] = e2[1] > 0 ? sqrt(e2[0] / e2[1]) : 0.0;
    }
    free(pidx); free(pval); free(pcnt);
    return 0;
}
