/*
 * Plain C oracle for the 255-bit number-theoretic transform.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference arm of bench.py may load this library.  It shares
 * no code with the CUDA library: its arithmetic is 4 x 64-bit limbs with
 * unsigned __int128 products and the textbook Montgomery multiplication of
 * Menezes-van Oorschot-Vanstone, Handbook of Applied Cryptography, Alg. 14.36
 * (radix b = 2^64), while the CUDA path works in 8 x 32-bit limbs.
 *
 * It computes the transform of MORPH Sec. 2.3.1 ("Number Theory
 * Transformation"), X_k = sum_n x_n omega_N^{kn} mod M, by the iterative
 * radix-2 Cooley-Tukey method (bit reversal, then log2 N butterfly stages),
 * plus the inverse (omega^-1, then N^-1) and the coset transform
 * (forward of x_n * s^n).  omega_N = g^((M-1)/N) with g the field's
 * multiplicative generator.  Elements are canonical, natural order,
 * 4 little-endian uint64 limbs each.
 *
 * Single-threaded by default: it is the reported CPU baseline "as it
 * stands".  oracle_set_threads(k) with k > 1 splits the butterflies of each
 * stage over k OpenMP threads (each thread takes a run of consecutive
 * butterflies and starts its twiddle at w^j by exponentiation); the
 * arithmetic and the results are the same.  That mode is the all-cores CPU
 * baseline.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int n_threads = 1;

typedef unsigned __int128 u128;

typedef struct {
    uint64_t m[4];     /* modulus, little-endian limbs */
    uint64_t mprime;   /* -m^{-1} mod 2^64 */
    uint64_t r1[4];    /* 2^256 mod m: Montgomery form of 1 */
    uint64_t r2[4];    /* 2^512 mod m */
    uint64_t g;        /* multiplicative generator */
    unsigned adicity;  /* 2-adicity of m - 1 */
} field_t;

static field_t FIELDS[2];
static int fields_ready = 0;

static const uint64_t MOD_BLS[4] = {0xffffffff00000001ULL, 0x53bda402fffe5bfeULL,
                                    0x3339d80809a1d805ULL, 0x73eda753299d7d48ULL};
static const uint64_t MOD_BN[4] = {0x43e1f593f0000001ULL, 0x2833e84879b97091ULL,
                                   0xb85045b68181585dULL, 0x30644e72e131a029ULL};

/* ------------------------------------------------------------ helpers */

static int geq(const uint64_t a[4], const uint64_t b[4]) {
    for (int i = 3; i >= 0; i--) {
        if (a[i] != b[i]) return a[i] > b[i];
    }
    return 1;
}

static void sub_raw(uint64_t r[4], const uint64_t a[4], const uint64_t b[4]) {
    uint64_t borrow = 0;
    for (int i = 0; i < 4; i++) {
        u128 d = (u128)a[i] - b[i] - borrow;
        r[i] = (uint64_t)d;
        borrow = (uint64_t)(d >> 64) ? 1 : 0;
    }
}

/* r = a + b mod m, a, b < m */
static void add_mod(const field_t *F, uint64_t r[4], const uint64_t a[4], const uint64_t b[4]) {
    uint64_t s[4];
    u128 c = 0;
    for (int i = 0; i < 4; i++) {
        c += (u128)a[i] + b[i];
        s[i] = (uint64_t)c;
        c >>= 64;
    }
    /* m < 2^255 for both fields, so a + b < 2^256: no carry out. */
    if (geq(s, F->m)) sub_raw(s, s, F->m);
    memcpy(r, s, sizeof s);
}

/* r = a - b mod m, a, b < m */
static void sub_mod(const field_t *F, uint64_t r[4], const uint64_t a[4], const uint64_t b[4]) {
    uint64_t d[4];
    if (geq(a, b)) {
        sub_raw(d, a, b);
    } else {
        uint64_t t[4];
        sub_raw(t, F->m, b);   /* m - b */
        u128 c = 0;
        for (int i = 0; i < 4; i++) {
            c += (u128)a[i] + t[i];
            d[i] = (uint64_t)c;
            c >>= 64;
        }
    }
    memcpy(r, d, sizeof d);
}

/* HAC Alg. 14.36: r = x * y * 2^-256 mod m, for x, y < m. */
static void mont_mul(const field_t *F, uint64_t r[4], const uint64_t x[4], const uint64_t y[4]) {
    uint64_t A[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 4; i++) {
        uint64_t u = (A[0] + x[i] * y[0]) * F->mprime;
        u128 c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)x[i] * y[j] + A[j];
            A[j] = (uint64_t)c;
            c >>= 64;
        }
        c += A[4];
        A[4] = (uint64_t)c;
        A[5] += (uint64_t)(c >> 64);
        c = 0;
        for (int j = 0; j < 4; j++) {
            c += (u128)u * F->m[j] + A[j];
            A[j] = (uint64_t)c;
            c >>= 64;
        }
        c += A[4];
        A[4] = (uint64_t)c;
        A[5] += (uint64_t)(c >> 64);
        /* A is now divisible by b: shift one limb down. */
        for (int j = 0; j < 5; j++) A[j] = A[j + 1];
        A[5] = 0;
    }
    uint64_t res[4] = {A[0], A[1], A[2], A[3]};
    if (A[4] || geq(res, F->m)) sub_raw(res, res, F->m);
    memcpy(r, res, sizeof res);
}

static void to_mont(const field_t *F, uint64_t r[4], const uint64_t a[4]) { mont_mul(F, r, a, F->r2); }

static void from_mont(const field_t *F, uint64_t r[4], const uint64_t a[4]) {
    static const uint64_t one[4] = {1, 0, 0, 0};
    mont_mul(F, r, a, one);
}

/* r = base^e (Montgomery form in and out), e given as 4 limbs. */
static void mont_pow(const field_t *F, uint64_t r[4], const uint64_t base[4], const uint64_t e[4]) {
    uint64_t acc[4], b[4];
    memcpy(acc, F->r1, sizeof acc);
    memcpy(b, base, sizeof b);
    for (int i = 0; i < 256; i++) {
        if ((e[i / 64] >> (i % 64)) & 1) mont_mul(F, acc, acc, b);
        mont_mul(F, b, b, b);
    }
    memcpy(r, acc, sizeof acc);
}

static void init_field(field_t *F, const uint64_t m[4], uint64_t g, unsigned adicity) {
    memcpy(F->m, m, sizeof F->m);
    F->g = g;
    F->adicity = adicity;
    /* Newton iteration for m0^{-1} mod 2^64 (m0 odd). */
    uint64_t inv = 1;
    for (int i = 0; i < 7; i++) inv *= 2 - m[0] * inv;
    F->mprime = (uint64_t)0 - inv;
    /* 2^256 mod m and 2^512 mod m by repeated doubling (m < 2^255). */
    uint64_t x[4] = {1, 0, 0, 0};
    for (int i = 0; i < 512; i++) {
        add_mod(F, x, x, x);
        if (i == 255) memcpy(F->r1, x, sizeof x);
    }
    memcpy(F->r2, x, sizeof x);
}

static void ensure_fields(void) {
    if (fields_ready) return;
    init_field(&FIELDS[0], MOD_BLS, 7, 32);
    init_field(&FIELDS[1], MOD_BN, 5, 28);
    fields_ready = 1;
}

/* omega_N = g^((m-1)/N), Montgomery form. */
static void root_mont(const field_t *F, unsigned log_n, uint64_t r[4]) {
    uint64_t e[4], g[4] = {F->g, 0, 0, 0}, gm[4];
    memcpy(e, F->m, sizeof e);
    e[0] -= 1;                              /* m is odd: no borrow */
    for (unsigned s = 0; s < log_n; s++) {  /* e >>= log_n */
        for (int i = 0; i < 4; i++) e[i] = (e[i] >> 1) | (i < 3 ? (e[i + 1] << 63) : 0);
    }
    to_mont(F, gm, g);
    mont_pow(F, r, gm, e);
}

static void inv_mont(const field_t *F, const uint64_t a_mont[4], uint64_t r[4]) {
    uint64_t e[4];
    memcpy(e, F->m, sizeof e);
    e[0] -= 2;
    mont_pow(F, r, a_mont, e);
}

/* One radix-2 stage (butterfly span len, twiddle root wl) with the n/2
 * butterflies t = block * len/2 + j split into runs over the threads; a run
 * starts its twiddle at wl^j (exponentiation) and steps it like the serial
 * loop, restarting at 1 where a new block begins. */
static void stage_threaded(const field_t *F, uint64_t (*a)[4], uint64_t n, uint64_t len, const uint64_t wl[4]) {
    const uint64_t half = len >> 1, total = n >> 1;
    const int64_t runs = (int64_t)(total < 4096 ? 1 : 4 * (uint64_t)n_threads);
#pragma omp parallel for schedule(static) num_threads(n_threads)
    for (int64_t r = 0; r < runs; r++) {
        const uint64_t t0 = total * (uint64_t)r / (uint64_t)runs, t1 = total * (uint64_t)(r + 1) / (uint64_t)runs;
        uint64_t wj[4];
        uint64_t e[4] = {t0 % half, 0, 0, 0};
        mont_pow(F, wj, wl, e);
        for (uint64_t t = t0; t < t1; t++) {
            const uint64_t j = t % half, i0 = (t / half) * len + j;
            if (j == 0) memcpy(wj, F->r1, sizeof wj);
            uint64_t u[4], v[4];
            memcpy(u, a[i0], sizeof u);
            mont_mul(F, v, a[i0 + half], wj);
            add_mod(F, a[i0], u, v);
            sub_mod(F, a[i0 + half], u, v);
            mont_mul(F, wj, wj, wl);
        }
    }
}

/* In-place iterative radix-2 DIT on Montgomery-form data with root w. */
static void radix2(const field_t *F, uint64_t (*a)[4], uint64_t n, unsigned log_n, const uint64_t w[4]) {
    for (uint64_t i = 0; i < n; i++) {
        uint64_t r = 0;
        for (unsigned b = 0; b < log_n; b++) r |= ((i >> b) & 1) << (log_n - 1 - b);
        if (r > i) {
            uint64_t t[4];
            memcpy(t, a[i], sizeof t);
            memcpy(a[i], a[r], sizeof t);
            memcpy(a[r], t, sizeof t);
        }
    }
    for (unsigned s = 1; s <= log_n; s++) {
        uint64_t len = (uint64_t)1 << s, half = len >> 1;
        uint64_t wl[4];
        /* w_len = w^(n/len): square w (log_n - s) times. */
        memcpy(wl, w, sizeof wl);
        for (unsigned k = s; k < log_n; k++) mont_mul(F, wl, wl, wl);
        if (n_threads > 1) {
            stage_threaded(F, a, n, len, wl);
            continue;
        }
        for (uint64_t start = 0; start < n; start += len) {
            uint64_t wj[4];
            memcpy(wj, F->r1, sizeof wj);
            for (uint64_t j = 0; j < half; j++) {
                uint64_t u[4], v[4];
                memcpy(u, a[start + j], sizeof u);
                mont_mul(F, v, a[start + j + half], wj);
                add_mod(F, a[start + j], u, v);
                sub_mod(F, a[start + j + half], u, v);
                mont_mul(F, wj, wj, wl);
            }
        }
    }
}

/*
 * kind: 0 forward, 1 inverse, 2 coset forward, 3 coset inverse
 *       (x_n = s^-n N^-1 sum_k X_k omega^-nk, the inverse of kind 2).
 * shift: coset shift s (4 limbs, canonical) or NULL for the generator.
 * in/out: n = 2^log_n elements of 4 limbs; in == out allowed.
 * Returns 0 on success, 1 bad field, 2 bad size, 3 bad kind, 4 no memory,
 * 5 an input is not canonical.
 */
int oracle_ntt(int field, int kind, unsigned log_n, const uint64_t *shift, const uint64_t *in, uint64_t *out) {
    ensure_fields();
    if (field < 0 || field > 1) return 1;
    const field_t *F = &FIELDS[field];
    if (log_n < 1 || log_n > F->adicity || log_n > 30) return 2;
    if (kind < 0 || kind > 3) return 3;
    uint64_t n = (uint64_t)1 << log_n;
    uint64_t (*a)[4] = (uint64_t(*)[4])malloc(n * 32);
    if (!a) return 4;
    uint64_t s_m[4], p[4];
    if (kind == 2 || kind == 3) {
        uint64_t s[4] = {F->g, 0, 0, 0};
        if (shift) memcpy(s, shift, sizeof s);
        to_mont(F, s_m, s);
        memcpy(p, F->r1, sizeof p);
    }
    for (uint64_t i = 0; i < n; i++) {
        if (geq(in + 4 * i, F->m)) {
            free(a);
            return 5;
        }
        to_mont(F, a[i], in + 4 * i);
        if (kind == 2) {
            mont_mul(F, a[i], a[i], p);
            mont_mul(F, p, p, s_m);
        }
    }
    uint64_t w[4];
    root_mont(F, log_n, w);
    if (kind == 1 || kind == 3) {
        uint64_t wi[4];
        inv_mont(F, w, wi);
        radix2(F, a, n, log_n, wi);
        uint64_t nn[4] = {n, 0, 0, 0}, nm[4], ninv[4];
        to_mont(F, nm, nn);
        inv_mont(F, nm, ninv);
        for (uint64_t i = 0; i < n; i++) mont_mul(F, a[i], a[i], ninv);
        if (kind == 3) {
            /* x_n *= s^-n */
            uint64_t si[4];
            inv_mont(F, s_m, si);
            for (uint64_t i = 0; i < n; i++) {
                mont_mul(F, a[i], a[i], p);
                mont_mul(F, p, p, si);
            }
        }
    } else {
        radix2(F, a, n, log_n, w);
    }
    for (uint64_t i = 0; i < n; i++) from_mont(F, out + 4 * i, a[i]);
    free(a);
    return 0;
}

/* out = sum_i coeffs[i] z^i (Horner), all canonical 4-limb values. */
int oracle_eval(int field, uint64_t n, const uint64_t *coeffs, const uint64_t *z, uint64_t *out) {
    ensure_fields();
    if (field < 0 || field > 1) return 1;
    const field_t *F = &FIELDS[field];
    uint64_t acc[4] = {0, 0, 0, 0}, zm[4], c[4];
    to_mont(F, zm, z);
    for (uint64_t i = n; i-- > 0;) {
        /* acc (standard) * z (Montgomery) -> standard */
        mont_mul(F, acc, acc, zm);
        memcpy(c, coeffs + 4 * i, sizeof c);
        add_mod(F, acc, acc, c);
    }
    memcpy(out, acc, sizeof acc);
    return 0;
}

/* out = omega_N (standard form). */
int oracle_root(int field, unsigned log_n, uint64_t *out) {
    ensure_fields();
    if (field < 0 || field > 1) return 1;
    const field_t *F = &FIELDS[field];
    if (log_n > F->adicity) return 2;
    uint64_t w[4];
    root_mont(F, log_n, w);
    from_mont(F, out, w);
    return 0;
}

/* out = a * b mod m (standard form in and out). */
int oracle_mul(int field, const uint64_t *a, const uint64_t *b, uint64_t *out) {
    ensure_fields();
    if (field < 0 || field > 1) return 1;
    const field_t *F = &FIELDS[field];
    uint64_t am[4];
    to_mont(F, am, a);
    mont_mul(F, out, am, b);
    return 0;
}

/* Threads for the butterfly stages of later oracle_ntt calls (1 = the plain
 * serial loop; 0 = every core OpenMP sees).  Returns the count now in use. */
int oracle_set_threads(int k) {
#ifdef _OPENMP
    if (k <= 0) k = omp_get_num_procs();
    n_threads = k;
#else
    (void)k;
    n_threads = 1;
#endif
    return n_threads;
}
