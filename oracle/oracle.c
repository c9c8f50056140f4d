/*
 * Dense FP64 CPU oracle for the 1-D nonuniform transforms of types 1, 2, 4, 5
 * and for the node-dependent quantities of the non-iterative inverse.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, calls or
 * includes this file; only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.  It shares no code, header, table or helper with
 * the CUDA path.
 *
 * Every routine here is the plain definition written out, in float64, with no
 * fast algorithm:
 *   - type-1 (Sec. II, Eq. 32):  A_k = sum_p a_p e^{-j 2 pi k t_p}
 *   - type-2 (Sec. II, Eq. 34):  s_p = sum_m S_m e^{+j 2 pi m t_p}
 *   - the type-2 system matrix G_{q,m} = e^{j 2 pi m t_q}; types 4 and 5
 *     (Eqs. 47 and 48) are solved from it by Gaussian elimination in the
 *     Python wrapper (the paper's GE benchmark, Sec. VI).
 *   - the Lagrange kernel L(z) = prod_p (z - z_p) (Eq. 11) at the shifted grid
 *     z_q = e^{j 2 pi (q/P + j a)} (the samples of Eq. 10), as an O(P^2)
 *     product;
 *   - L'(z_p) = prod_{q != p} (z_p - z_q), the derivative samples of Sec. III-D,
 *     as an O(P^2) product;
 *   - the node weights of Eqs. 27 and 40:
 *       w_p = h(-P t_p + j P a) / (L'(z_p) z_p),  h(t) = 1/(e^{j 2 pi t} - 1)  (Eq. 17).
 *
 * Phases are exact: a node is carried as the 64-bit fixed-point fraction
 * T = t * 2^64, so e^{j 2 pi m t} is computed from the integer m*T mod 2^64
 * and the only rounding left is one libm sin/cos of an argument in [-pi, pi).
 *
 * Products over P factors are accumulated as sums of logarithms (magnitude)
 * and of turns reduced modulo 1 (argument), so they neither overflow nor lose
 * the phase to a large unreduced sum.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define TWO_PI 6.283185307179586476925286766559

/* Node canonicalisation: t = x/(2 pi) mod 1 in [0,1), T = trunc(t * 2^64). */
void oracle_canon(int64_t n, const double* x, uint64_t* T, double* t)
{
    for (int64_t i = 0; i < n; ++i) {
        double u = x[i] / TWO_PI;
        u -= floor(u);
        if (u >= 1.0) u = 0.0;
        T[i] = (uint64_t)(u * 18446744073709551616.0);
        if (t) t[i] = u;
    }
}

/* phase fraction of an exact 64-bit turn count, in [-1/2, 1/2) */
static inline double turns(uint64_t ph)
{
    return (double)(int64_t)ph * 5.42101086242752217003726400434970855712890625e-20; /* 2^-64 */
}

static inline void cis_turns(uint64_t ph, double sign, double* re, double* im)
{
    double ang = TWO_PI * turns(ph);
    *re = cos(ang);
    *im = sign * sin(ang);
}

/* Type-1, Eq. 32: A_k = sum_p a_p e^{-j 2 pi k t_p}, k = k0 .. k0+M-1.
   a, A interleaved complex128. */
void oracle_type1(int64_t P, const uint64_t* T, const double* a,
                  int64_t k0, int64_t M, double* A)
{
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < M; ++k) {
        uint64_t kk = (uint64_t)(k0 + k);
        double sr = 0.0, si = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            double cr, ci;
            cis_turns(kk * T[p], -1.0, &cr, &ci);
            double ar = a[2 * p], ai = a[2 * p + 1];
            sr += ar * cr - ai * ci;
            si += ar * ci + ai * cr;
        }
        A[2 * k] = sr;
        A[2 * k + 1] = si;
    }
}

/* Type-2, Eq. 34: s_q = sum_m S_m e^{+j 2 pi (m0+m) t_q}, m = 0 .. M-1,
   at Q nodes. */
void oracle_type2(int64_t M, int64_t m0, const double* S,
                  int64_t Q, const uint64_t* T, double* s)
{
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < Q; ++q) {
        double sr = 0.0, si = 0.0;
        for (int64_t m = 0; m < M; ++m) {
            double cr, ci;
            cis_turns((uint64_t)(m0 + m) * T[q], 1.0, &cr, &ci);
            double br = S[2 * m], bi = S[2 * m + 1];
            sr += br * cr - bi * ci;
            si += br * ci + bi * cr;
        }
        s[2 * q] = sr;
        s[2 * q + 1] = si;
    }
}

/* Type-2 system matrix of Eq. 48, row-major: G[q][m] = e^{j 2 pi m t_q}. */
void oracle_matrix(int64_t P, const uint64_t* T, double* G)
{
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < P; ++q)
        for (int64_t m = 0; m < P; ++m)
            cis_turns((uint64_t)m * T[q], 1.0, &G[2 * (q * P + m)], &G[2 * (q * P + m) + 1]);
}

/* Accumulator for a product of complex factors: log-magnitude plus
   argument in turns kept reduced to [-1/2, 1/2). */
typedef struct { double logmag, turn; } prodacc;

static inline void prod_mul(prodacc* acc, double re, double im)
{
    acc->logmag += log(hypot(re, im));
    acc->turn += atan2(im, re) / TWO_PI;
    acc->turn -= nearbyint(acc->turn);
}

static inline void prod_out(const prodacc* acc, double* re, double* im)
{
    double m = exp(acc->logmag);
    double ang = TWO_PI * acc->turn;
    *re = m * cos(ang);
    *im = m * sin(ang);
}

/* Kernel samples of Eq. 10: K_q = L(z_q) = prod_p (z_q - z_p),
   z_q = rho e^{j 2 pi q/P} (rho = e^{-2 pi a}), z_p = e^{j 2 pi t_p}. */
void oracle_kernel_samples(int64_t P, const uint64_t* T, double rho, double* K)
{
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < P; ++q) {
        double ang = TWO_PI * (double)q / (double)P;
        double zr = rho * cos(ang), zi = rho * sin(ang);
        prodacc acc = {0.0, 0.0};
        for (int64_t p = 0; p < P; ++p) {
            double cr, ci;
            cis_turns(T[p], 1.0, &cr, &ci);
            prod_mul(&acc, zr - cr, zi - ci);
        }
        prod_out(&acc, &K[2 * q], &K[2 * q + 1]);
    }
}

/* Derivative samples of Sec. III-D: D_p = L'(z_p) = prod_{q != p} (z_p - z_q).
   Each factor is formed from the exact phase difference:
   z_p - z_q = z_p (1 - e^{j 2 pi (t_q - t_p)}). */
void oracle_deriv_samples(int64_t P, const uint64_t* T, double* D)
{
    #pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        prodacc acc = {0.0, 0.0};
        double zpr, zpi;
        cis_turns(T[p], 1.0, &zpr, &zpi);
        for (int64_t q = 0; q < P; ++q) {
            if (q == p) continue;
            double er, ei;
            cis_turns(T[q] - T[p], 1.0, &er, &ei);
            double fr = 1.0 - er, fi = -ei;          /* 1 - e^{j2pi(t_q-t_p)} */
            prod_mul(&acc, zpr * fr - zpi * fi, zpr * fi + zpi * fr);
        }
        prod_out(&acc, &D[2 * p], &D[2 * p + 1]);
    }
}

/* Node weights of Eqs. 27 / 40:
   w_p = h(-P t_p + j P a) / (L'(z_p) z_p),  h(t) = 1/(e^{j 2 pi t} - 1),
   h(-P t_p + j P a) = 1 / (rho^P e^{-j 2 pi P t_p} - 1).
   D = L'(z_p) as returned by oracle_deriv_samples. */
void oracle_weights(int64_t P, const uint64_t* T, double rho, const double* D, double* w)
{
    double rP = pow(rho, (double)P);
    for (int64_t p = 0; p < P; ++p) {
        double er, ei, zr, zi;
        cis_turns((uint64_t)P * T[p], -1.0, &er, &ei);     /* e^{-j 2 pi P t_p} */
        cis_turns(T[p], 1.0, &zr, &zi);                      /* z_p */
        double hr = rP * er - 1.0, hi = rP * ei;             /* 1/h */
        double dr = D[2 * p] * zr - D[2 * p + 1] * zi;       /* L'(z_p) z_p */
        double di = D[2 * p] * zi + D[2 * p + 1] * zr;
        double br = hr * dr - hi * di, bi = hr * di + hi * dr;   /* denominator */
        double nn = br * br + bi * bi;
        w[2 * p] = br / nn;
        w[2 * p + 1] = -bi / nn;
    }
}

/* Type-1, Eq. 32, at an arbitrary list of integer frequencies ks[0..nk-1]. */
void oracle_type1_at(int64_t P, const uint64_t* T, const double* a, int64_t nk, const int64_t* ks, double* A)
{
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nk; ++i) {
        uint64_t kk = (uint64_t)ks[i];
        double sr = 0.0, si = 0.0;
        for (int64_t p = 0; p < P; ++p) {
            double cr, ci;
            cis_turns(kk * T[p], -1.0, &cr, &ci);
            double ar = a[2 * p], ai = a[2 * p + 1];
            sr += ar * cr - ai * ci;
            si += ar * ci + ai * cr;
        }
        A[2 * i] = sr;
        A[2 * i + 1] = si;
    }
}

/* Type-2, Eq. 34, with the coefficients at an arbitrary list of integer
   frequencies ms[0..nm-1]: s_q = sum_i S_i e^{+j 2 pi ms[i] t_q} at Q nodes. */
void oracle_type2_at(int64_t nm, const int64_t* ms, const double* S, int64_t Q, const uint64_t* T, double* s)
{
    #pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < Q; ++q) {
        double sr = 0.0, si = 0.0;
        for (int64_t i = 0; i < nm; ++i) {
            double cr, ci;
            cis_turns((uint64_t)ms[i] * T[q], 1.0, &cr, &ci);
            double br = S[2 * i], bi = S[2 * i + 1];
            sr += br * cr - bi * ci;
            si += br * ci + bi * cr;
        }
        s[2 * q] = sr;
        s[2 * q + 1] = si;
    }
}
