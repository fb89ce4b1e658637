/*
 * FP64 CPU oracle for random-circuit amplitudes -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load
 * this file's library.  It shares no code with the GPU library.
 *
 * What it computes (paper Sec. 2, "RQC simulation methods"): the state-vector
 * method -- the n-qubit state as 2^n complex amplitudes, evolved gate by gate
 * from |0...0>, then read at the queried bitstrings, amp(x) = <x|U|0^n>.
 * The tensor-network contraction of the paper reaches exactly this value (up
 * to rounding) once every slice is summed (Sec. 3.1, sub-networks from broken
 * edges).  A single slice -- one fixed value b of a broken wire -- is the same
 * evolution with the projector |b><b| applied to that wire right after the
 * gate that produces it; the sum over b of those projectors is the identity,
 * which is why the slices sum to the whole.
 *
 * Conventions (the paper is silent; readings recorded in the design notes):
 *   - state index i, qubit q <-> bit q of i (little endian);
 *   - a 4x4 gate is row-major over |q0 q1>, q0 the high bit of the 2-bit
 *     local index; a 2x2 gate is row-major (out, in).
 *
 * Also here: the brute-force reference (product of full 2^n x 2^n unitaries,
 * each gate embedded by its definition -- no strided updates), used to pin
 * the state-vector code at small n.
 */
#include <complex.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

int oracle_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* |0...0> */
static void sv_init(int n, cplx *psi) {
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i) psi[i] = 0.0;
    psi[0] = 1.0;
}

/* single-qubit gate g (2x2, row-major) on qubit q */
static void sv_apply_1q(int n, cplx *psi, int q, const cplx g[4]) {
    const int64_t half = (int64_t)1 << (n - 1);
    const int64_t low = ((int64_t)1 << q) - 1;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < half; ++t) {
        /* insert a 0 at bit q */
        const int64_t i0 = ((t & ~low) << 1) | (t & low);
        const int64_t i1 = i0 | ((int64_t)1 << q);
        const cplx a0 = psi[i0], a1 = psi[i1];
        psi[i0] = g[0] * a0 + g[1] * a1;
        psi[i1] = g[2] * a0 + g[3] * a1;
    }
}

/* two-qubit gate g (4x4 over |q0 q1>, q0 high bit) on qubits q0, q1 */
static void sv_apply_2q(int n, cplx *psi, int q0, int q1, const cplx g[16]) {
    const int64_t quarter = (int64_t)1 << (n - 2);
    const int lo = q0 < q1 ? q0 : q1, hi = q0 < q1 ? q1 : q0;
    const int64_t mlo = ((int64_t)1 << lo) - 1;
    const int64_t mhi = ((int64_t)1 << hi) - 1;
    const int64_t b0 = (int64_t)1 << q0, b1 = (int64_t)1 << q1;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < quarter; ++t) {
        /* insert zeros at bit positions lo then hi */
        int64_t i = ((t & ~mlo) << 1) | (t & mlo);
        i = ((i & ~mhi) << 1) | (i & mhi);
        const int64_t idx[4] = {i, i | b1, i | b0, i | b0 | b1}; /* local 2*x0+x1 */
        cplx a[4];
        for (int l = 0; l < 4; ++l) a[l] = psi[idx[l]];
        for (int r = 0; r < 4; ++r) {
            cplx s = 0.0;
            for (int c = 0; c < 4; ++c) s += g[4 * r + c] * a[c];
            psi[idx[r]] = s;
        }
    }
}

/* projector |v><v| on qubit q: zero every amplitude whose bit q differs */
static void sv_project(int n, cplx *psi, int q, int v) {
    const int64_t dim = (int64_t)1 << n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < dim; ++i)
        if (((i >> q) & 1) != v) psi[i] = 0.0;
}

static void load_gate(const double *re, const double *im, int g, int two, cplx *m) {
    const int cnt = two ? 16 : 4;
    for (int k = 0; k < cnt; ++k) {
        /* 1q gates are stored in the top-left 2x2 of a 4x4 row-major block */
        const int src = two ? k : (k / 2) * 4 + (k % 2);
        m[k] = re[16 * g + src] + I * im[16 * g + src];
    }
}

/*
 * Evolve |0^n> through gates 0..n_gates-1.  After gate g (and before gate 0
 * when proj_after == -1) apply every projector with proj_after == g.
 * state: 2^n complex doubles (interleaved re, im), written.
 * Returns 0, or -1 on a bad argument.
 */
int oracle_sv_run(int n, int n_gates, const int32_t *q0, const int32_t *q1,
                  const double *mre, const double *mim,
                  int n_proj, const int32_t *proj_q, const int32_t *proj_after,
                  const int32_t *proj_val, double *state) {
    if (n < 2 || n > 34) return -1;
    cplx *psi = (cplx *)state;
    sv_init(n, psi);
    for (int p = 0; p < n_proj; ++p)
        if (proj_after[p] == -1) sv_project(n, psi, proj_q[p], proj_val[p]);
    for (int g = 0; g < n_gates; ++g) {
        cplx m[16];
        if (q0[g] < 0 || q0[g] >= n || q1[g] >= n || q1[g] == q0[g]) return -1;
        if (q1[g] < 0) {
            load_gate(mre, mim, g, 0, m);
            sv_apply_1q(n, psi, q0[g], m);
        } else {
            load_gate(mre, mim, g, 1, m);
            sv_apply_2q(n, psi, q0[g], q1[g], m);
        }
        for (int p = 0; p < n_proj; ++p)
            if (proj_after[p] == g) sv_project(n, psi, proj_q[p], proj_val[p]);
    }
    return 0;
}

/*
 * Read the queried amplitudes: out[j] = state[x(j)] where x(j) has
 * fixed_bits[q] on every non-open qubit and bit t of j on open_qubits[t].
 */
void oracle_gather(int n, const double *state, int n_open, const int32_t *open_qubits,
                   const uint8_t *fixed_bits, double *out) {
    const cplx *psi = (const cplx *)state;
    cplx *o = (cplx *)out;
    int64_t base = 0;
    int is_open[64] = {0};
    for (int t = 0; t < n_open; ++t) is_open[open_qubits[t]] = 1;
    for (int q = 0; q < n; ++q)
        if (!is_open[q] && fixed_bits[q]) base |= (int64_t)1 << q;
    const int64_t cnt = (int64_t)1 << n_open;
    for (int64_t j = 0; j < cnt; ++j) {
        int64_t x = base;
        for (int t = 0; t < n_open; ++t)
            if ((j >> t) & 1) x |= (int64_t)1 << open_qubits[t];
        o[j] = psi[x];
    }
}

/*
 * Brute force, n <= 10: U = U_{G-1} ... U_0 with each U_g the full 2^n x 2^n
 * matrix of gate g, built entry by entry from its definition
 *   U_g[x][y] = m[l(x)][l(y)] if x and y agree off the gate's qubits, else 0,
 * where l(.) is the gate-local index.  Returns column 0 of U = U|0^n>.
 * Cost O(G * 8^n): meant for n <= 8.
 */
int oracle_bruteforce(int n, int n_gates, const int32_t *q0, const int32_t *q1,
                      const double *mre, const double *mim, double *out_col0) {
    if (n < 1 || n > 10) return -1;
    const int64_t d = (int64_t)1 << n;
    cplx *U = (cplx *)calloc((size_t)(d * d), sizeof(cplx));
    cplx *G = (cplx *)calloc((size_t)(d * d), sizeof(cplx));
    cplx *T = (cplx *)calloc((size_t)(d * d), sizeof(cplx));
    if (!U || !G || !T) { free(U); free(G); free(T); return -2; }
    for (int64_t i = 0; i < d; ++i) U[i * d + i] = 1.0;
    for (int g = 0; g < n_gates; ++g) {
        const int two = q1[g] >= 0;
        cplx m[16];
        load_gate(mre, mim, g, two, m);
        int64_t gmask = (int64_t)1 << q0[g];
        if (two) gmask |= (int64_t)1 << q1[g];
        for (int64_t x = 0; x < d; ++x)
            for (int64_t y = 0; y < d; ++y) {
                cplx v = 0.0;
                if ((x & ~gmask) == (y & ~gmask)) {
                    if (two) {
                        const int lx = 2 * (int)((x >> q0[g]) & 1) + (int)((x >> q1[g]) & 1);
                        const int ly = 2 * (int)((y >> q0[g]) & 1) + (int)((y >> q1[g]) & 1);
                        v = m[4 * lx + ly];
                    } else {
                        const int lx = (int)((x >> q0[g]) & 1), ly = (int)((y >> q0[g]) & 1);
                        v = m[2 * lx + ly];
                    }
                }
                G[x * d + y] = v;
            }
        /* T = G * U */
#pragma omp parallel for schedule(static)
        for (int64_t r = 0; r < d; ++r)
            for (int64_t c = 0; c < d; ++c) {
                cplx s = 0.0;
                for (int64_t k = 0; k < d; ++k) s += G[r * d + k] * U[k * d + c];
                T[r * d + c] = s;
            }
        cplx *sw = U; U = T; T = sw;
    }
    cplx *o = (cplx *)out_col0;
    for (int64_t r = 0; r < d; ++r) o[r] = U[r * d + 0];
    free(U); free(G); free(T);
    return 0;
}
