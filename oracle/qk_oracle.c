/*
 * Reference state-vector simulator in complex128 -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and bench.py's CPU-baseline leg may load this
 * library.  It shares no code with the CUDA path and is written to be read
 * against the definitions, not to be fast: one plain loop per operation, sums in
 * index order, double precision throughout.
 *
 * Conventions (the paper's command scripts, Appendix A):
 *   - the state of n qubits is 2^n complex amplitudes psi[i], stored as
 *     interleaved doubles (re, im); qubit q is bit q of the index i;
 *   - in a target list the first-listed qubit is the most significant bit of the
 *     register value (so "SigmaX nQ-1" sets the work register to 1);
 *   - controls act when every control qubit is |1>.
 *
 * Every function returns 0 on success and -1 on invalid arguments (the state is
 * then untouched), except orc_measure which returns the outcome bit.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define ORC_MAX_QUBITS 40
#define ORC_MAX_K 10
#define ORC_PI 3.14159265358979323846

static int bad_qubit_list(int n, const int *q, int k)
{
    for (int a = 0; a < k; ++a) {
        if (q[a] < 0 || q[a] >= n) return 1;
        for (int b = 0; b < a; ++b)
            if (q[a] == q[b]) return 1;
    }
    return 0;
}

/* Register value of index i over targets t[0..k-1], t[0] the MSB. */
static uint64_t register_value(uint64_t i, const int *t, int k)
{
    uint64_t x = 0;
    for (int a = 0; a < k; ++a)
        x = (x << 1) | ((i >> t[a]) & 1u);
    return x;
}

/* Index i with the register over t[0..k-1] overwritten by value x. */
static uint64_t with_register(uint64_t i, const int *t, int k, uint64_t x)
{
    for (int a = 0; a < k; ++a) {
        uint64_t bit = (x >> (k - 1 - a)) & 1u;
        i = (i & ~(1ull << t[a])) | (bit << t[a]);
    }
    return i;
}

static int controls_hold(uint64_t i, const int *c, int nc)
{
    for (int a = 0; a < nc; ++a)
        if (((i >> c[a]) & 1u) == 0) return 0;
    return 1;
}

/*
 * Controlled k-qubit unitary (gate operation on k targets, Q-Kit section: single,
 * entangling and multi-qubit gates, and gates defined as a matrix).
 * u is the 2^k x 2^k matrix, row-major, interleaved (re, im); row/column index is
 * the register value over targets (targets[0] = MSB).  For every group of 2^k
 * amplitudes that share the non-target bits and whose control bits are all 1, the
 * group vector v (indexed by register value) is replaced by u v.
 */
int orc_apply_unitary(double *psi_d, int n, int k, const int *targets, const double *u,
                      const int *controls, int nc)
{
    if (n < 0 || n > ORC_MAX_QUBITS || k < 1 || k > ORC_MAX_K || k > n || nc < 0) return -1;
    if (bad_qubit_list(n, targets, k) || bad_qubit_list(n, controls, nc)) return -1;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < nc; ++b)
            if (targets[a] == controls[b]) return -1;

    cplx *psi = (cplx *)psi_d;
    const uint64_t dim = 1ull << n, g = 1ull << k;
    uint64_t tmask = 0;
    for (int a = 0; a < k; ++a) tmask |= 1ull << targets[a];
    int failed = 0;

    /* Groups are independent: the all-core build (-fopenmp, for timing the
     * oracle on every host core) splits them across threads, each with its own
     * scratch; every group's arithmetic and summation order are unchanged.  The
     * plain build ignores the pragmas and runs the loop as written. */
#ifdef _OPENMP
#pragma omp parallel reduction(| : failed)
#endif
    {
        cplx *v = malloc(sizeof(cplx) * g), *w = malloc(sizeof(cplx) * g);
        if (!v || !w) failed = 1;
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (uint64_t base = 0; base < dim; ++base) {
            if (!v || !w) continue;
            if (base & tmask) continue;                 /* one visit per group */
            if (!controls_hold(base, controls, nc)) continue;
            for (uint64_t x = 0; x < g; ++x) v[x] = psi[with_register(base, targets, k, x)];
            for (uint64_t r = 0; r < g; ++r) {
                cplx s = 0;
                for (uint64_t c = 0; c < g; ++c)
                    s += CMPLX(u[2 * (r * g + c)], u[2 * (r * g + c) + 1]) * v[c];
                w[r] = s;
            }
            for (uint64_t x = 0; x < g; ++x) psi[with_register(base, targets, k, x)] = w[x];
        }
        free(v);
        free(w);
    }
    return failed ? -1 : 0;
}

/*
 * Gate defined as a function (Q-Kit section: custom gates "as a function", the
 * oracle gate): a permutation f of the w-bit register value.  Where every control
 * is |1>, the amplitude at register value x moves to register value f(x); elsewhere
 * nothing moves.  f must be a bijection of [0, 2^w) (checked).
 */
int orc_apply_perm(double *psi_d, int n, int w, const int *targets, const uint64_t *f,
                   const int *controls, int nc)
{
    if (n < 0 || n > ORC_MAX_QUBITS || w < 1 || w > n || w > 30 || nc < 0) return -1;
    if (bad_qubit_list(n, targets, w) || bad_qubit_list(n, controls, nc)) return -1;
    for (int a = 0; a < w; ++a)
        for (int b = 0; b < nc; ++b)
            if (targets[a] == controls[b]) return -1;
    const uint64_t g = 1ull << w;
    unsigned char *seen = calloc(g, 1);
    if (!seen) return -1;
    for (uint64_t x = 0; x < g; ++x) {
        if (f[x] >= g || seen[f[x]]) { free(seen); return -1; }
        seen[f[x]] = 1;
    }
    free(seen);

    cplx *psi = (cplx *)psi_d;
    const uint64_t dim = 1ull << n;
    cplx *out = malloc(sizeof(cplx) * dim);
    if (!out) return -1;
    for (uint64_t i = 0; i < dim; ++i) {
        uint64_t dst = i;
        if (controls_hold(i, controls, nc))
            dst = with_register(i, targets, w, f[register_value(i, targets, w)]);
        out[dst] = psi[i];
    }
    memcpy(psi, out, sizeof(cplx) * dim);
    free(out);
    return 0;
}

/*
 * QuModExpUaj (Appendix A): x -> c x mod N on the w-qubit register when x < N,
 * x unchanged when x >= N (the paper is silent there; identity keeps the map a
 * permutation).  The caller passes c = a^(2^j) mod N; gcd(c, N) must be 1.
 * The product is formed in 128-bit arithmetic, so any N < 2^w <= 2^30 is exact.
 */
int orc_apply_mulmod(double *psi_d, int n, int w, const int *targets, uint64_t c, uint64_t N,
                     const int *controls, int nc)
{
    if (w < 1 || w > 30 || N < 2 || N > (1ull << w) || c >= N) return -1;
    uint64_t g = 1ull << w;
    uint64_t *f = malloc(sizeof(uint64_t) * g);
    if (!f) return -1;
    for (uint64_t x = 0; x < g; ++x)
        f[x] = (x < N) ? (uint64_t)(((unsigned __int128)c * x) % N) : x;
    int rc = orc_apply_perm(psi_d, n, w, targets, f, controls, nc);
    free(f);
    return rc;
}

/* Probability that qubit q reads 0: sum of |psi_i|^2 over i with bit q = 0, in index order. */
double orc_prob0(const double *psi_d, int n, int q)
{
    const cplx *psi = (const cplx *)psi_d;
    double p0 = 0.0;
    for (uint64_t i = 0; i < (1ull << n); ++i)
        if (((i >> q) & 1u) == 0) {
            p0 += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
        }
    return p0;
}

/*
 * In-place measurement of one qubit (Q-Kit section; Measure in Appendix A).
 * Outcome m = 0 iff u < P0 (the project's sampling rule; the paper only says the
 * outcome follows the Born probabilities).  The other branch is zeroed and the
 * kept branch is scaled by 1/sqrt(P_m).  *p0_out receives P0.  Returns m, or -1.
 */
int orc_measure(double *psi_d, int n, int q, double u, double *p0_out)
{
    if (n < 1 || n > ORC_MAX_QUBITS || q < 0 || q >= n) return -1;
    cplx *psi = (cplx *)psi_d;
    double p0 = orc_prob0(psi_d, n, q);
    int m = (u < p0) ? 0 : 1;
    double pm = p0;
    if (m == 1) {
        /* recompute P1 directly rather than as 1 - P0 */
        pm = 0.0;
        for (uint64_t i = 0; i < (1ull << n); ++i)
            if ((i >> q) & 1u)
                pm += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    }
    double scale = (pm > 0.0) ? 1.0 / sqrt(pm) : 0.0;
    for (uint64_t i = 0; i < (1ull << n); ++i) {
        if ((int)((i >> q) & 1u) == m) psi[i] *= scale;
        else psi[i] = 0.0;
    }
    if (p0_out) *p0_out = p0;
    return m;
}

/*
 * Semiclassical phase correction "RPhase 0,-e..-1" (Appendix A, nx2n branch):
 * the |1> component of the target is multiplied by exp(i theta) with
 *   theta = -2 pi * sum_{l=1..e} m_l / 2^(l+1),
 * m_l the l-th listed classical bit (most recent stage first).  This is the
 * inverse-QFT rotation of iterative phase estimation (Kitaev / Griffiths-Niu).
 */
int orc_apply_rphase(double *psi_d, int n, int target, const unsigned char *mbits, int e)
{
    if (n < 1 || n > ORC_MAX_QUBITS || target < 0 || target >= n || e < 0 || e > 62) return -1;
    double frac = 0.0;
    for (int l = 1; l <= e; ++l)
        if (mbits[l - 1]) frac += ldexp(1.0, -(l + 1));
    cplx f = cexp(CMPLX(0.0, -2.0 * ORC_PI * frac));
    cplx *psi = (cplx *)psi_d;
    for (uint64_t i = 0; i < (1ull << n); ++i)
        if ((i >> target) & 1u) psi[i] *= f;
    return 0;
}

/* Squared 2-norm, summed in index order. */
double orc_norm2(const double *psi_d, int n)
{
    const cplx *psi = (const cplx *)psi_d;
    double s = 0.0;
    for (uint64_t i = 0; i < (1ull << n); ++i)
        s += creal(psi[i]) * creal(psi[i]) + cimag(psi[i]) * cimag(psi[i]);
    return s;
}
