/*
 * FP64 CPU oracle for damped dynamic relaxation of truss (fiber) networks.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the plain, slow, obviously correct
 * statement of what the GPU library computes. Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it. It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Method (Merson & Shephard, "Using Hierarchical Parallelism to Accelerate the
 * Solution of Many Small Partial Differential Equations", Algorithm 1): a
 * static equilibrium problem is mapped onto damped explicit central-difference
 * dynamics and iterated until the force residual, not the time, has converged
 * (Section III). Every step below follows Algorithm 1 in the paper's order, in
 * serial element-scatter form and in the caller's node order.
 *
 * Readings of what the paper leaves open (the paper prints no force law,
 * mass, time step, damping, norm or stress formula):
 *   force     N_e = EA_e (l_e / L_e - 1), axial along the current element;
 *             node a gets +(N/l) d, node b gets -(N/l) d, d = x_b - x_a
 *   mass      lumped, element density rho*A_e = EA_e / L_e^2, half of the
 *             element mass rho*A_e*L_e = EA_e/L_e to each end node
 *   time step alpha * min_e L_e sqrt(rho*A_e / EA_e); with the mass above the
 *             axial tangent EA/L bounds every element frequency, so the step is
 *             the same every iteration (it is alpha)
 *   damping   f_d = -c m v with the half-step velocity, c per RVE
 *   residual  r = ||g_free||_2, converged when r <= tol * f_ref with
 *             f_ref = max(||g(F X)||_2, ||g(x0)||_2) over all DOFs
 *   init      0: u = 0 on free nodes, (F - I) X on fixed nodes;
 *             1: u = (F - I) X everywhere; 2: free u given (warm), fixed (F-I)X
 *   stress    sigma = (1/V) sum_e (N_e/l_e) d_e (x) d_e, V = det(F) V0
 *   loop      repeat ... until: at least one iteration runs
 *
 * Each function cites the part of the paper it follows. None of them is
 * blocked, fused or reordered beyond Algorithm 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_NAN = 2, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

/* Reference lengths L_e = |X_b - X_a| (Algorithm 1, "load mesh and compute
 * edge connectivity"). */
void oracle_ref_lengths(int64_t E, const double *X, const int32_t *el, double *L) {
    for (int64_t e = 0; e < E; ++e) {
        const double *xa = X + 3 * (int64_t)el[2 * e], *xb = X + 3 * (int64_t)el[2 * e + 1];
        double dx = xb[0] - xa[0], dy = xb[1] - xa[1], dz = xb[2] - xa[2];
        L[e] = sqrt(dx * dx + dy * dy + dz * dz);
    }
}

/* Lumped mass by element integration (Algorithm 1, "compute mass matrix"):
 * rho*A_e = EA_e / L_e^2, element mass rho*A_e*L_e split equally. */
void oracle_masses(int64_t n, int64_t E, const int32_t *el, const double *EA, const double *L,
                   double *m) {
    for (int64_t i = 0; i < n; ++i) m[i] = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        double rhoA = EA[e] / (L[e] * L[e]);
        double me = rhoA * L[e];
        m[el[2 * e]] += 0.5 * me;
        m[el[2 * e + 1]] += 0.5 * me;
    }
}

/* Critical step of an axial element with the lumped masses above, times the
 * safety factor alpha (Algorithm 1, "compute next time step"). */
double oracle_time_step(int64_t E, const double *EA, const double *L, double alpha) {
    double dtc = INFINITY;
    for (int64_t e = 0; e < E; ++e) {
        double rhoA = EA[e] / (L[e] * L[e]);
        double t = L[e] * sqrt(rhoA / EA[e]);
        if (t < dtc) dtc = t;
    }
    return alpha * dtc;
}

/* Internal nodal forces g(x) (Algorithm 1, getInternalForces): zero, then
 * scatter each element's axial force to its two nodes, as the paper's naive
 * path does (Section III). */
void oracle_internal_forces(int64_t n, const double *x, int64_t E, const int32_t *el,
                            const double *EA, const double *L, double *g) {
    for (int64_t i = 0; i < 3 * n; ++i) g[i] = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        int64_t a = el[2 * e], b = el[2 * e + 1];
        double d0 = x[3 * b] - x[3 * a], d1 = x[3 * b + 1] - x[3 * a + 1],
               d2 = x[3 * b + 2] - x[3 * a + 2];
        double l = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double N = EA[e] * (l / L[e] - 1.0);
        double q = N / l;
        g[3 * a] += q * d0; g[3 * a + 1] += q * d1; g[3 * a + 2] += q * d2;
        g[3 * b] -= q * d0; g[3 * b + 1] -= q * d1; g[3 * b + 2] -= q * d2;
    }
}

/* Strain energy W = sum_e 1/2 EA_e L_e (l_e/L_e - 1)^2, whose negative
 * gradient is the internal force above. */
double oracle_strain_energy(int64_t n, const double *x, int64_t E, const int32_t *el,
                            const double *EA, const double *L) {
    (void)n;
    double W = 0.0;
    for (int64_t e = 0; e < E; ++e) {
        int64_t a = el[2 * e], b = el[2 * e + 1];
        double d0 = x[3 * b] - x[3 * a], d1 = x[3 * b + 1] - x[3 * a + 1],
               d2 = x[3 * b + 2] - x[3 * a + 2];
        double l = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double s = l / L[e] - 1.0;
        W += 0.5 * EA[e] * L[e] * s * s;
    }
    return W;
}

static double det3(const double *F) {
    return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
           F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* Volume-averaged Cauchy stress in the current configuration (the quantity
 * the microscale returns to the macroscale, Section I):
 * sigma = (1/V) sum_e (N_e / l_e) d_e (x) d_e, V = det(F) V0. Row-major. */
void oracle_stress_virial(int64_t n, const double *x, int64_t E, const int32_t *el,
                          const double *EA, const double *L, const double *F, double V0,
                          double *sigma) {
    (void)n;
    double s[9] = {0};
    for (int64_t e = 0; e < E; ++e) {
        int64_t a = el[2 * e], b = el[2 * e + 1];
        double d[3] = {x[3 * b] - x[3 * a], x[3 * b + 1] - x[3 * a + 1], x[3 * b + 2] - x[3 * a + 2]};
        double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double q = EA[e] * (l / L[e] - 1.0) / l;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) s[3 * r + c] += q * d[r] * d[c];
    }
    double V = det3(F) * V0;
    for (int k = 0; k < 9; ++k) sigma[k] = s[k] / V;
}

/* The same stress from the boundary reactions: with g the internal force,
 * sum_e t_e (x) d_e = -sum_i g_i (x) x_i, which at equilibrium only the fixed
 * nodes contribute to. Not symmetric away from equilibrium. */
void oracle_stress_boundary(int64_t n, const double *x, const double *g, const uint8_t *fixed,
                            const double *F, double V0, double *sigma) {
    double s[9] = {0};
    for (int64_t i = 0; i < n; ++i) {
        if (!fixed[i]) continue;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) s[3 * r + c] -= g[3 * i + r] * x[3 * i + c];
    }
    double V = det3(F) * V0;
    for (int k = 0; k < 9; ++k) sigma[k] = s[k] / V;
}

static double norm2(int64_t n, const double *g, const uint8_t *mask, int want) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (mask && mask[i] != want) continue;
        s += g[3 * i] * g[3 * i] + g[3 * i + 1] * g[3 * i + 1] + g[3 * i + 2] * g[3 * i + 2];
    }
    return sqrt(s);
}

/*
 * Algorithm 1 for one RVE.
 *
 * In : n, X (n*3), E, el (E*2, node ids), EA (E), fixed (n), F (9, row-major),
 *      c (damping), tol, max_iter (>= 1), alpha (time-step safety factor),
 *      init (0 reference, 1 affine, 2 warm), u_warm (n*3, used when init = 2),
 *      V0, want_ke (1: track kinetic energy; 2: also the internal and
 *      external work of the energy balance check).
 * Out: u (n*3, displacement at the last force evaluation), sigma (9),
 *      iters, rel_res (r / f_ref, 0 when f_ref = 0), f_ref, ke (last KE or 0),
 *      wint, wext (work since the start, 0 unless want_ke = 2; may be NULL).
 *
 * Energy balance (Algorithm 1, "optionally check energy balance": three
 * reductions over the free DOFs per iteration). With du = dt v^(n-1/2) the
 * step's displacement increment and f_d = -c m v^(n-1/2) the damping force:
 *   kinetic   K    = 1/2 sum m |v^n|^2 (full-step velocity)
 *   internal  Wint = Wint - 1/2 sum du . (g^(n-1) + g^n)   (energy stored;
 *             g is the net internal force on a node, so -g resists)
 *   external  Wext = Wext + 1/2 sum du . (f_d^(n-1) + f_d^n)  (work of the
 *             damping forces; the prescribed nodes do not move while the
 *             iteration runs, so their reactions do no work)
 * trapezoidal in du, with g^0 the initial force and f_d^0 = 0.
 * Returns ORC_OK, ORC_MAXITER, ORC_NAN, or a negative error.
 */
int oracle_dr_solve(int64_t n, const double *X, int64_t E, const int32_t *el, const double *EA,
                    const uint8_t *fixed, const double *F, double c, double tol, int64_t max_iter,
                    double alpha, int init, const double *u_warm, double V0, int want_ke,
                    double *u, double *sigma, int64_t *iters, double *rel_res, double *f_ref_out,
                    double *ke_out, double *wint_out, double *wext_out) {
    if (n <= 0 || E < 0 || max_iter < 1) return ORC_EINVAL;
    double *L = malloc(sizeof(double) * (E ? E : 1));
    double *m = malloc(sizeof(double) * n);
    double *x = malloc(sizeof(double) * 3 * n);
    double *v = calloc(3 * n, sizeof(double));
    double *a = calloc(3 * n, sizeof(double));
    double *g = malloc(sizeof(double) * 3 * n);
    uint8_t *fx = malloc(n);
    double *gp = want_ke == 2 ? calloc(3 * n, sizeof(double)) : NULL;   /* g^(n-1) */
    double *fdp = want_ke == 2 ? calloc(3 * n, sizeof(double)) : NULL;  /* f_d^(n-1) */
    if (!L || !m || !x || !v || !a || !g || !fx || (want_ke == 2 && (!gp || !fdp))) {
        free(L); free(m); free(x); free(v); free(a); free(g); free(fx); free(gp); free(fdp);
        return ORC_ENOMEM;
    }

    /* Algorithm 1: load mesh, connectivity (given), mass matrix. A free node
     * that no element touches has no mass and no force: it is held fixed. */
    oracle_ref_lengths(E, X, el, L);
    oracle_masses(n, E, el, EA, L, m);
    for (int64_t i = 0; i < n; ++i) fx[i] = (uint8_t)(fixed[i] || m[i] == 0.0);
    fixed = fx;

    /* f_ref part 1: the affine configuration x = F X over all DOFs. */
    for (int64_t i = 0; i < n; ++i)
        for (int r = 0; r < 3; ++r)
            x[3 * i + r] = F[3 * r] * X[3 * i] + F[3 * r + 1] * X[3 * i + 1] + F[3 * r + 2] * X[3 * i + 2];
    oracle_internal_forces(n, x, E, el, EA, L, g);
    double f_aff = norm2(n, g, NULL, 0);

    /* Algorithm 1: displacement boundary conditions on fixed nodes, initial
     * displacement of the free nodes. */
    for (int64_t i = 0; i < n; ++i) {
        for (int r = 0; r < 3; ++r) {
            double uaff = x[3 * i + r] - X[3 * i + r];
            if (fixed[i] || init == 1) u[3 * i + r] = uaff;
            else if (init == 2) u[3 * i + r] = u_warm[3 * i + r];
            else u[3 * i + r] = 0.0;
        }
    }
    for (int64_t k = 0; k < 3 * n; ++k) x[k] = X[k] + u[k];

    /* Algorithm 1: getInternalForces(u); update accelerations (free DOFs). */
    oracle_internal_forces(n, x, E, el, EA, L, g);
    double f0 = norm2(n, g, NULL, 0);
    double f_ref = f_aff > f0 ? f_aff : f0;
    for (int64_t i = 0; i < n; ++i)
        if (!fixed[i])
            for (int r = 0; r < 3; ++r) a[3 * i + r] = g[3 * i + r] / m[i];
    if (want_ke == 2)
        for (int64_t k = 0; k < 3 * n; ++k) gp[k] = g[k];

    int status = ORC_MAXITER;
    int64_t it = 0;
    double r_norm = 0.0, ke = 0.0, wint = 0.0, wext = 0.0;
    for (;;) {
        /* compute next time step */
        double dt = oracle_time_step(E, EA, L, alpha);
        /* partial velocity update; update displacements (free DOFs) */
        for (int64_t i = 0; i < n; ++i) {
            if (fixed[i]) continue;
            for (int r = 0; r < 3; ++r) {
                v[3 * i + r] += 0.5 * dt * a[3 * i + r];
                u[3 * i + r] += dt * v[3 * i + r];
                x[3 * i + r] = X[3 * i + r] + u[3 * i + r];
            }
        }
        /* getInternalForces(u) */
        oracle_internal_forces(n, x, E, el, EA, L, g);
        /* damping force; force residual (free-DOF reduction); update
         * accelerations; partial velocity update */
        double rs = 0.0, wi = 0.0, we = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            if (fixed[i]) continue;
            for (int r = 0; r < 3; ++r) {
                double fd = -c * m[i] * v[3 * i + r];
                if (want_ke == 2) {
                    /* energy check: this step's increment times the forces at
                     * its two ends (v still holds v^(n-1/2) here) */
                    double du = dt * v[3 * i + r];
                    wi += du * (gp[3 * i + r] + g[3 * i + r]);
                    we += du * (fdp[3 * i + r] + fd);
                    gp[3 * i + r] = g[3 * i + r];
                    fdp[3 * i + r] = fd;
                }
                rs += g[3 * i + r] * g[3 * i + r];
                a[3 * i + r] = (g[3 * i + r] + fd) / m[i];
                v[3 * i + r] += 0.5 * dt * a[3 * i + r];
            }
        }
        r_norm = sqrt(rs);
        wint -= 0.5 * wi;
        wext += 0.5 * we;
        /* optional energy check: kinetic part */
        if (want_ke) {
            ke = 0.0;
            for (int64_t i = 0; i < n; ++i)
                if (!fixed[i])
                    ke += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                                        v[3 * i + 2] * v[3 * i + 2]);
        }
        /* update iteration count; until force residual converged */
        ++it;
        if (!isfinite(r_norm)) { status = ORC_NAN; break; }
        if (r_norm <= tol * f_ref) { status = ORC_OK; break; }
        if (it >= max_iter) { status = ORC_MAXITER; break; }
    }

    oracle_stress_virial(n, x, E, el, EA, L, F, V0, sigma);
    *iters = it;
    *rel_res = f_ref > 0.0 ? r_norm / f_ref : (r_norm > 0.0 ? INFINITY : 0.0);
    *f_ref_out = f_ref;
    *ke_out = ke;
    if (wint_out) *wint_out = wint;
    if (wext_out) *wext_out = wext;
    free(L); free(m); free(x); free(v); free(a); free(g); free(fx); free(gp); free(fdp);
    return status;
}

/* ---------------------------------------------------------------------------
 * Brute-force static equilibrium by Newton's method on tiny networks.
 * Independent of the dynamics: solves g_free(x) = 0 directly with the
 * consistent tangent K_e = (EA/L) n (x) n + (N/l) (I - n (x) n), assembled
 * densely and factored by LU with partial pivoting.
 * ------------------------------------------------------------------------- */

static int lu_solve(int64_t N, double *A, double *b) {
    for (int64_t k = 0; k < N; ++k) {
        int64_t p = k;
        double best = fabs(A[k * N + k]);
        for (int64_t i = k + 1; i < N; ++i)
            if (fabs(A[i * N + k]) > best) { best = fabs(A[i * N + k]); p = i; }
        if (best == 0.0) return -1;
        if (p != k) {
            for (int64_t j = 0; j < N; ++j) {
                double t = A[k * N + j]; A[k * N + j] = A[p * N + j]; A[p * N + j] = t;
            }
            double t = b[k]; b[k] = b[p]; b[p] = t;
        }
        for (int64_t i = k + 1; i < N; ++i) {
            double f = A[i * N + k] / A[k * N + k];
            if (f == 0.0) continue;
            for (int64_t j = k; j < N; ++j) A[i * N + j] -= f * A[k * N + j];
            b[i] -= f * b[k];
        }
    }
    for (int64_t k = N - 1; k >= 0; --k) {
        double s = b[k];
        for (int64_t j = k + 1; j < N; ++j) s -= A[k * N + j] * b[j];
        b[k] = s / A[k * N + k];
    }
    return 0;
}

/*
 * Newton iterations from x = X + u (u in/out, fixed DOFs untouched).
 * Returns the number of iterations (>= 0) or -1 if the tangent is singular.
 * last_step gets the max-norm of the last correction.
 */
int oracle_newton(int64_t n, const double *X, int64_t E, const int32_t *el, const double *EA,
                  const uint8_t *fixed, double *u, int max_it, double step_tol, double *last_step) {
    int64_t *dof = malloc(sizeof(int64_t) * n);
    int64_t nf = 0;
    for (int64_t i = 0; i < n; ++i) dof[i] = fixed[i] ? -1 : nf++;
    int64_t N = 3 * nf;
    double *L = malloc(sizeof(double) * (E ? E : 1));
    double *x = malloc(sizeof(double) * 3 * n);
    double *g = malloc(sizeof(double) * 3 * n);
    double *K = malloc(sizeof(double) * (N ? N * N : 1));
    double *rhs = malloc(sizeof(double) * (N ? N : 1));
    oracle_ref_lengths(E, X, el, L);
    int it = 0, rc = 0;
    *last_step = 0.0;
    for (; it < max_it; ++it) {
        for (int64_t k = 0; k < 3 * n; ++k) x[k] = X[k] + u[k];
        oracle_internal_forces(n, x, E, el, EA, L, g);
        memset(K, 0, sizeof(double) * (N ? N * N : 1));
        for (int64_t e = 0; e < E; ++e) {
            int64_t na = el[2 * e], nb = el[2 * e + 1];
            double d[3] = {x[3 * nb] - x[3 * na], x[3 * nb + 1] - x[3 * na + 1], x[3 * nb + 2] - x[3 * na + 2]};
            double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double nv[3] = {d[0] / l, d[1] / l, d[2] / l};
            double k_ax = EA[e] / L[e], q = EA[e] * (l / L[e] - 1.0) / l;
            double Ke[9];
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s)
                    Ke[3 * r + s] = k_ax * nv[r] * nv[s] + q * ((r == s ? 1.0 : 0.0) - nv[r] * nv[s]);
            /* dg_a/dx_a = -Ke, dg_a/dx_b = +Ke, dg_b/dx_a = +Ke, dg_b/dx_b = -Ke */
            int64_t da = dof[na], db = dof[nb];
            for (int r = 0; r < 3; ++r)
                for (int s = 0; s < 3; ++s) {
                    double kv = Ke[3 * r + s];
                    if (da >= 0) K[(3 * da + r) * N + 3 * da + s] -= kv;
                    if (db >= 0) K[(3 * db + r) * N + 3 * db + s] -= kv;
                    if (da >= 0 && db >= 0) {
                        K[(3 * da + r) * N + 3 * db + s] += kv;
                        K[(3 * db + r) * N + 3 * da + s] += kv;
                    }
                }
        }
        for (int64_t i = 0; i < n; ++i)
            if (dof[i] >= 0)
                for (int r = 0; r < 3; ++r) rhs[3 * dof[i] + r] = -g[3 * i + r];
        if (lu_solve(N, K, rhs) != 0) { rc = -1; break; }
        double mx = 0.0;
        for (int64_t i = 0; i < n; ++i)
            if (dof[i] >= 0)
                for (int r = 0; r < 3; ++r) {
                    double du = rhs[3 * dof[i] + r];
                    u[3 * i + r] += du;
                    if (fabs(du) > mx) mx = fabs(du);
                }
        *last_step = mx;
        if (mx <= step_tol) { ++it; break; }
    }
    free(dof); free(L); free(x); free(g); free(K); free(rhs);
    return rc < 0 ? -1 : it;
}
