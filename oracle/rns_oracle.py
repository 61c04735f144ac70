"""Plain CPU oracle of the paper's RNS lazy modular multiplication.

TEST INFRASTRUCTURE ONLY (same rule as ``ntt_oracle``): only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline / reference arm of
``bench.py`` use it.  It shares no code with the CUDA library: its own prime
search, its own constant tables, Python big integers throughout.

What it computes (MORPH, Sec. 3.2.3-3.2.4 and Alg. 1, "MXU RNS Lazy"): a
product x * y of elements of the prime field F_M carried out in a larger
non-prime residue number system, with the reduction modulo M turned into a
small matrix product over bytes.  Alg. 1 is partly garbled (its CRT factor
is written with the wrong modulus and its output is stated as an exact
equation although the reduction is lazy), so the steps below are this
module's reading of it; every reading is listed in the design notes.

Two bases of 31-bit primes: Q = prod q_i (i < I) and P = prod p_j (j < J).
An element is carried as its residues in base Q, as an integer in [0, L)
with L = (sum_i q_i + I) * M ("lazy": congruent to the field element, not
reduced).  Q > 4 L^2, so the product of two such integers is exact in base
Q, and P > 2^20 L.

  1. VecMul          c_i  = x_i y_i mod q_i                      (c = x y exactly)
  2. CRT digits      xi_i = c_i (Q/q_i)^-1 mod q_i
  3. quotient        v = sum_i xi_i f_i, f_i = ceil(2^u / q_i);  k = floor(v / 2^u)
                     (k = floor(sum_i xi_i / q_i), the CRT quotient, exactly)
  4. ByteDecompose   xi_i = sum_b xi_{i,b} 2^(8b)
  5. Einsum          acc_{j,h} = sum_{i,b} xi_{i,b} E1[i,b,j,h]     (8-bit x 8-bit)
                     E1[i,b,j,h] = byte h of (2^(8b) ((Q/q_i) mod M) (P/p_j)^-1 mod p_j)
  6. ByteMerge       s_j = sum_h acc_{j,h} 2^(8h)
  7. correction      eta_j = (s_j + k g_j) mod p_j,  g_j = (M - (Q mod M)) (P/p_j)^-1 mod p_j
     so eta_j = R (P/p_j)^-1 mod p_j for
         R = sum_i xi_i ((Q/q_i) mod M) + k (M - (Q mod M))  ==  x y  (mod M),
     0 <= R < L.
  8-11. the same four steps take R from base P back to base Q exactly (a
     base extension, no reduction mod M): v2, k2 from eta and
     f'_j = ceil(2^u / p_j); acc2_{i,h} = sum_{j,b} eta_{j,b} E2[j,b,i,h],
     E2[j,b,i,h] = byte h of (2^(8b) (P/p_j) mod q_i);
     r_i = (sum_h acc2_{i,h} 2^(8h) + k2 g2_i) mod q_i,  g2_i = (-P) mod q_i.

The output r (R's residues in base Q) is again a lazy element, so
products chain.  Pins (tests/test_rns_oracle.py): R == x y (mod M) and
0 <= R < L against big-integer arithmetic; k and k2 equal the exact CRT
quotients; long chains; the extreme inputs L - 1; planted mistakes.
"""

from __future__ import annotations

from dataclasses import dataclass

from .ntt_oracle import get_field

U_SHIFT = 58            # 2^u scaling of the quotient estimates (both bases)


def _is_prime_u32(n: int) -> bool:
    """Deterministic Miller-Rabin for n < 2^32 (bases 2, 7, 61)."""
    if n < 2:
        return False
    for p in (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37, 41, 43, 47, 53, 59, 61):
        if n % p == 0:
            return n == p
    d, s = n - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in (2, 7, 61):
        x = pow(a, d, n)
        if x in (1, n - 1):
            continue
        for _ in range(s - 1):
            x = x * x % n
            if x == n - 1:
                break
        else:
            return False
    return True


def _primes_below(start: int):
    n = start - 1
    while n > 2:
        if _is_prime_u32(n):
            yield n
        n -= 1


def _prod(v) -> int:
    out = 1
    for x in v:
        out *= x
    return out


@dataclass(frozen=True)
class RnsBasis:
    modulus: int        # M
    q: tuple            # base Q moduli
    p: tuple            # base P moduli
    L: int              # lazy bound: elements are integers in [0, L)

    @property
    def Q(self) -> int:
        return _prod(self.q)

    @property
    def P(self) -> int:
        return _prod(self.p)


def rns_basis(field) -> RnsBasis:
    """Base Q: the largest primes below 2^31, as few as give Q > 4 L^2 with
    L = (sum q + I) M; base P: the next primes below them, as few as give
    P > 2^20 L."""
    M = get_field(field).modulus
    gen = _primes_below(1 << 31)
    q = []
    while True:
        q.append(next(gen))
        L = (sum(q) + len(q)) * M
        if _prod(q) > 4 * L * L:
            break
    p = []
    while _prod(p) <= (L << 20):
        p.append(next(gen))
    return RnsBasis(M, tuple(q), tuple(p), L)


def to_rns(x: int, mods) -> list[int]:
    return [x % m for m in mods]


def from_rns(r, mods) -> int:
    """CRT reconstruction (the integer in [0, prod mods))."""
    Mall = _prod(mods)
    x = 0
    for ri, m in zip(r, mods):
        Mi = Mall // m
        x += ri * Mi * pow(Mi, -1, m)
    return x % Mall


def byte_decompose(v: int, nbytes: int = 4) -> list[int]:
    return [(v >> (8 * b)) & 0xFF for b in range(nbytes)]


def byte_merge(parts) -> int:
    return sum(int(v) << (8 * h) for h, v in enumerate(parts))


def tables(basis: RnsBasis) -> dict:
    """Constants of the two conversions (E1, g, f for Q -> P; E2, g2, f2 for
    P -> Q), written out from their definitions."""
    M, q, p = basis.modulus, basis.q, basis.p
    Q, P = basis.Q, basis.P
    I, J = len(q), len(p)
    q_hat_inv = [pow(Q // qi, -1, qi) for qi in q]
    p_hat_inv = [pow(P // pj, -1, pj) for pj in p]
    E1 = [[[[0] * 4 for _ in range(J)] for _ in range(4)] for _ in range(I)]
    for i in range(I):
        w = (Q // q[i]) % M
        for b in range(4):
            for j in range(J):
                val = ((w << (8 * b)) * p_hat_inv[j]) % p[j]
                E1[i][b][j] = byte_decompose(val)
    g = [((M - Q % M) * p_hat_inv[j]) % p[j] for j in range(J)]
    E2 = [[[[0] * 4 for _ in range(I)] for _ in range(4)] for _ in range(J)]
    for j in range(J):
        for b in range(4):
            for i in range(I):
                E2[j][b][i] = byte_decompose(((P // p[j]) << (8 * b)) % q[i])
    g2 = [(-P) % q[i] for i in range(I)]
    f = [-(-(1 << U_SHIFT) // qi) for qi in q]      # ceil(2^u / q_i)
    f2 = [-(-(1 << U_SHIFT) // pj) for pj in p]
    return {"q_hat_inv": q_hat_inv, "E1": E1, "g": g, "f": f, "E2": E2, "g2": g2, "f2": f2}


def rns_mul_lazy(basis: RnsBasis, x, y, tabs: dict | None = None, trace: dict | None = None) -> list[int]:
    """One lazy product: x, y are residue lists in base Q of integers in
    [0, L); returns the residues in base Q of R, R == x y (mod M), R < L."""
    t = tables(basis) if tabs is None else tabs
    q, p = basis.q, basis.p
    I, J = len(q), len(p)
    # 1-2. element-wise products and CRT digits
    c = [x[i] * y[i] % q[i] for i in range(I)]
    xi = [c[i] * t["q_hat_inv"][i] % q[i] for i in range(I)]
    # 3. quotient estimate
    v = sum(xi[i] * t["f"][i] for i in range(I))
    k = v >> U_SHIFT
    # 4-6. byte decomposition, byte product, byte merge
    xb = [byte_decompose(xi[i]) for i in range(I)]
    eta = []
    for j in range(J):
        acc = [sum(xb[i][b] * t["E1"][i][b][j][h] for i in range(I) for b in range(4)) for h in range(4)]
        # 7. correction and residue
        eta.append((byte_merge(acc) + k * t["g"][j]) % p[j])
    # 8-11. exact extension back to base Q
    v2 = sum(eta[j] * t["f2"][j] for j in range(J))
    k2 = v2 >> U_SHIFT
    eb = [byte_decompose(eta[j]) for j in range(J)]
    r = []
    for i in range(I):
        acc2 = [sum(eb[j][b] * t["E2"][j][b][i][h] for j in range(J) for b in range(4)) for h in range(4)]
        r.append((byte_merge(acc2) + k2 * t["g2"][i]) % q[i])
    if trace is not None:
        trace.update(c=c, xi=xi, k=k, eta=eta, k2=k2)
    return r
