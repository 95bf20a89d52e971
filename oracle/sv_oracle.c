/*
 * sv_oracle.c -- the CPU oracle of the state-vector path (TEST INFRASTRUCTURE).
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load or run this file. The product path (the CUDA library) never does, and
 * this file shares no code, header or table with it.
 *
 * What it computes: exact state-vector simulation in complex128, written as the
 * plain definitions (Sec. II: the state is a complex vector of 2^n amplitudes
 * and the simulation is exact; Sec. II-C: index bit q is qubit q):
 *
 *   orc_apply        gate application with a dense 2^k x 2^k matrix and optional
 *                    controls (Table I, "Gate application"), one group of 2^k
 *                    amplitudes at a time, no structure exploited;
 *   orc_expect_pauli <psi| P |psi> for a Pauli string P (Table I, "Expectation"):
 *                    apply each single-site Pauli matrix to a copy of psi, then
 *                    take the inner product;
 *   orc_parity_probs probabilities of even/odd parity of a set of qubits, i.e.
 *                    a measurement in the Z-product basis (Table I, "Measurement");
 *   orc_collapse     collapse onto one parity outcome and renormalise
 *                    (Table I: probability and collapse are separate);
 *   orc_norm2        sum of |psi_i|^2;
 *   orc_pauli_rotation  psi <- exp(i theta P) psi = cos(theta) psi + i sin(theta) P psi
 *                    (Table I, "Pauli rotation"), P applied site by site;
 *   orc_sample       measurement outcomes without collapse (Table I, "Sampler"):
 *                    for each r in [0, 1) the basis index i with
 *                    cum(i-1) <= r * cum(N-1) < cum(i), cum(i) = sum_{k<=i} |psi_k|^2.
 *
 * Conventions where the paper is silent: the row/column index bit j of a gate
 * matrix belongs to targets[j]; matrices are row-major; a control holds when
 * its qubit equals its control value (1 if none given).
 *
 * Amplitudes and matrix entries are passed as interleaved (re, im) doubles,
 * which C99 lays out exactly like `double complex`.
 *
 * Parity is pinned by tests/test_oracle.py (closed forms, brute force, numpy).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex zc;

#define ORC_OK 0
#define ORC_BAD_ARG 1
#define ORC_NO_MEM 2

int orc_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    return omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

/* offset of group member j: bit t of j placed at qubit targets[t] */
static uint64_t member_offset(uint64_t j, const int *targets, int k)
{
    uint64_t off = 0;
    for (int t = 0; t < k; ++t)
        if ((j >> t) & 1u) off |= 1ull << targets[t];
    return off;
}

static int check_qubits(int n, const int *targets, int k, const int *controls, int c)
{
    if (n < 1 || n > 40 || k < 1 || k > 6 || c < 0 || k + c > n) return ORC_BAD_ARG;
    uint64_t seen = 0;
    for (int t = 0; t < k + c; ++t) {
        int q = t < k ? targets[t] : controls[t - k];
        if (q < 0 || q >= n || ((seen >> q) & 1u)) return ORC_BAD_ARG;
        seen |= 1ull << q;
    }
    return ORC_OK;
}

/*
 * psi <- G psi, G = M on targets where the controls hold, identity elsewhere.
 * Every index i whose target bits are all 0 and whose control bits hold is the
 * first member of one group; the group's amplitudes are gathered, multiplied by
 * M and written back.
 */
int orc_apply(double *psi_ri, int n, const int *targets, int k,
              const int *controls, const int *control_values, int c,
              const double *matrix_ri)
{
    if (check_qubits(n, targets, k, controls, c) != ORC_OK) return ORC_BAD_ARG;
    zc *psi = (zc *)psi_ri;
    const zc *M = (const zc *)matrix_ri;
    const uint64_t N = 1ull << n;
    const uint64_t D = 1ull << k;
    uint64_t tmask = 0, cmask = 0, cwant = 0;
    for (int t = 0; t < k; ++t) tmask |= 1ull << targets[t];
    for (int t = 0; t < c; ++t) {
        cmask |= 1ull << controls[t];
        if (control_values == NULL || control_values[t] != 0) cwant |= 1ull << controls[t];
    }
    uint64_t off[64];
    for (uint64_t j = 0; j < D; ++j) off[j] = member_offset(j, targets, k);

    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < (int64_t)N; ++i) {
        uint64_t base = (uint64_t)i;
        if (base & tmask) continue;
        if ((base & cmask) != cwant) continue;
        zc in[64], out[64];
        for (uint64_t l = 0; l < D; ++l) in[l] = psi[base | off[l]];
        for (uint64_t j = 0; j < D; ++j) {
            zc acc = 0;
            for (uint64_t l = 0; l < D; ++l) acc += M[j * D + l] * in[l];
            out[j] = acc;
        }
        for (uint64_t j = 0; j < D; ++j) psi[base | off[j]] = out[j];
    }
    return ORC_OK;
}

/* The three Pauli matrices, row-major, by code 1 = X, 2 = Y, 3 = Z (0 = I). */
static void pauli_matrix(int code, zc m[4])
{
    switch (code) {
    case 1: m[0] = 0; m[1] = 1;  m[2] = 1; m[3] = 0;  break;  /* X = [[0,1],[1,0]]   */
    case 2: m[0] = 0; m[1] = -I; m[2] = I; m[3] = 0;  break;  /* Y = [[0,-i],[i,0]]  */
    case 3: m[0] = 1; m[1] = 0;  m[2] = 0; m[3] = -1; break;  /* Z = [[1,0],[0,-1]]  */
    default: m[0] = 1; m[1] = 0; m[2] = 0; m[3] = 1;  break;
    }
}

/*
 * out = <psi| P |psi> (complex; its imaginary part is zero up to rounding
 * because P is Hermitian). P = prod_s paulis[s] acting on qubit sites[s].
 */
int orc_expect_pauli(const double *psi_ri, int n, const int *paulis, const int *sites,
                     int n_sites, double *out_ri)
{
    if (n < 1 || n > 40 || n_sites < 0) return ORC_BAD_ARG;
    uint64_t seen = 0;
    for (int s = 0; s < n_sites; ++s) {
        if (sites[s] < 0 || sites[s] >= n || paulis[s] < 0 || paulis[s] > 3) return ORC_BAD_ARG;
        if ((seen >> sites[s]) & 1u) return ORC_BAD_ARG;
        seen |= 1ull << sites[s];
    }
    const uint64_t N = 1ull << n;
    const zc *psi = (const zc *)psi_ri;
    zc *phi = (zc *)malloc(N * sizeof(zc));
    if (!phi) return ORC_NO_MEM;
    memcpy(phi, psi, N * sizeof(zc));
    for (int s = 0; s < n_sites; ++s) {
        if (paulis[s] == 0) continue;
        zc m[4];
        pauli_matrix(paulis[s], m);
        int tq = sites[s];
        orc_apply((double *)phi, n, &tq, 1, NULL, NULL, 0, (const double *)m);
    }
    zc acc = 0;
    for (uint64_t i = 0; i < N; ++i) acc += conj(psi[i]) * phi[i];
    free(phi);
    out_ri[0] = creal(acc);
    out_ri[1] = cimag(acc);
    return ORC_OK;
}

/* parity of the measured qubits in basis index i */
static int parity_of(uint64_t i, const int *qubits, int m)
{
    int p = 0;
    for (int t = 0; t < m; ++t) p ^= (int)((i >> qubits[t]) & 1u);
    return p;
}

/* probs[0] = sum of |psi_i|^2 over even parity, probs[1] over odd parity */
int orc_parity_probs(const double *psi_ri, int n, const int *qubits, int m, double *probs)
{
    if (n < 1 || n > 40 || m < 1 || m > n) return ORC_BAD_ARG;
    for (int t = 0; t < m; ++t)
        if (qubits[t] < 0 || qubits[t] >= n) return ORC_BAD_ARG;
    const zc *psi = (const zc *)psi_ri;
    double p[2] = {0.0, 0.0};
    for (uint64_t i = 0; i < (1ull << n); ++i) {
        double a = cabs(psi[i]);
        p[parity_of(i, qubits, m)] += a * a;
    }
    probs[0] = p[0];
    probs[1] = p[1];
    return ORC_OK;
}

/* keep the amplitudes whose parity equals `outcome`, scale them by 1/sqrt(prob) */
int orc_collapse(double *psi_ri, int n, const int *qubits, int m, int outcome, double prob)
{
    if (n < 1 || n > 40 || m < 1 || m > n || (outcome != 0 && outcome != 1) || !(prob > 0.0))
        return ORC_BAD_ARG;
    zc *psi = (zc *)psi_ri;
    const double scale = 1.0 / sqrt(prob);
    for (uint64_t i = 0; i < (1ull << n); ++i)
        psi[i] = parity_of(i, qubits, m) == outcome ? psi[i] * scale : 0.0;
    return ORC_OK;
}

double orc_norm2(const double *psi_ri, int n)
{
    const zc *psi = (const zc *)psi_ri;
    double acc = 0.0;
    for (uint64_t i = 0; i < (1ull << n); ++i) {
        double a = cabs(psi[i]);
        acc += a * a;
    }
    return acc;
}

/* psi <- cos(theta) psi + i sin(theta) P psi, P = prod_s paulis[s] on qubit sites[s] */
int orc_pauli_rotation(double *psi_ri, int n, const int *paulis, const int *sites, int n_sites, double theta)
{
    if (n < 1 || n > 40 || n_sites < 0) return ORC_BAD_ARG;
    uint64_t seen = 0;
    for (int s = 0; s < n_sites; ++s) {
        if (sites[s] < 0 || sites[s] >= n || paulis[s] < 0 || paulis[s] > 3) return ORC_BAD_ARG;
        if ((seen >> sites[s]) & 1u) return ORC_BAD_ARG;
        seen |= 1ull << sites[s];
    }
    const uint64_t N = 1ull << n;
    zc *psi = (zc *)psi_ri;
    zc *phi = (zc *)malloc(N * sizeof(zc));
    if (!phi) return ORC_NO_MEM;
    memcpy(phi, psi, N * sizeof(zc));
    for (int s = 0; s < n_sites; ++s) {
        if (paulis[s] == 0) continue;
        zc m[4];
        pauli_matrix(paulis[s], m);
        int tq = sites[s];
        orc_apply((double *)phi, n, &tq, 1, NULL, NULL, 0, (const double *)m);
    }
    const double c = cos(theta), sn = sin(theta);
    for (uint64_t i = 0; i < N; ++i) psi[i] = c * psi[i] + I * sn * phi[i];
    free(phi);
    return ORC_OK;
}

/* out[t] = smallest i with r_t * cum(N-1) < cum(i) */
int orc_sample(const double *psi_ri, int n, const double *randnums, int n_samples, int64_t *out)
{
    if (n < 1 || n > 40 || n_samples < 0) return ORC_BAD_ARG;
    const uint64_t N = 1ull << n;
    const zc *psi = (const zc *)psi_ri;
    double *cum = (double *)malloc(N * sizeof(double));
    if (!cum) return ORC_NO_MEM;
    double acc = 0.0;
    for (uint64_t i = 0; i < N; ++i) {
        double a = cabs(psi[i]);
        acc += a * a;
        cum[i] = acc;
    }
    for (int t = 0; t < n_samples; ++t) {
        if (!(randnums[t] >= 0.0 && randnums[t] < 1.0)) {
            free(cum);
            return ORC_BAD_ARG;
        }
        const double target = randnums[t] * acc;
        uint64_t lo = 0, hi = N - 1;          /* first index with cum > target */
        while (lo < hi) {
            uint64_t mid = lo + (hi - lo) / 2;
            if (cum[mid] > target) hi = mid; else lo = mid + 1;
        }
        out[t] = (int64_t)lo;
    }
    free(cum);
    return ORC_OK;
}
