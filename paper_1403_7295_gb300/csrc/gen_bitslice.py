#!/usr/bin/env python3
"""Generate aes_bitslice_circuit.cuh: the AES S-box and inverse S-box as
straight-line Boolean circuits (AND / XOR / NOT) on bit-slice words.

Route (FIPS-197 §5.1.1 defines SubBytes as inversion in GF(2^8) followed by
an affine map; the inversion is computed here in a tower of fields):

  GF(4)   = GF(2)[W] / (W^2 + W + 1)
  GF(16)  = GF(4)[Z] / (Z^2 + Z + mu),      mu = W or W^2
  GF(256) = GF(16)[Y] / (Y^2 + Y + lam),    lam: a GF(16) constant making
                                            the polynomial irreducible
  inverse of h*Y + l:  d = (h^2*lam + h*l + l^2)^-1,  result (h*d)*Y + (h+l)*d
  inverse in GF(16) the same way over GF(4); inverse in GF(4) = squaring.

An isomorphism T from the AES polynomial basis to the tower basis maps x to
a root beta of x^8 + x^4 + x^3 + x + 1 in the tower field.  Then
  S(x)    = A . T^-1 . inv(T . x) + 0x63
  S^-1(y) = T^-1 . inv(T . A^-1 . (y + 0x63))
with A the affine matrix.  Every signal is tracked as a set of "atoms"
(input bits and AND outputs) combined by XOR.  The XOR networks between AND
layers are built as short linear programs with the distance-based greedy
heuristic of Boyar and Peralta: each new XOR is the sum of two signals
already built that most reduces the total distance of the layer's targets
(the distance of a target being how many built signals must still be added
to reach it; exact, from a table over the layer's span).  The whole circuit
is evaluated on all 256 inputs before anything is written.

The choice of mu, lam and beta changes the gate count; PARAMS holds, for each
direction, the choice with the fewest gates over all of them (found by
`python gen_bitslice.py --search`, about two minutes).

Usage: python gen_bitslice.py   (writes aes_bitslice_circuit.cuh beside itself)
"""
from __future__ import annotations

import os
import sys

import numpy as np

AES_POLY = 0x11B

# ---------------------------------------------------------------- fields ----


def aes_mul(a: int, b: int) -> int:
    p = 0
    while b:
        if b & 1:
            p ^= a
        a <<= 1
        if a & 0x100:
            a ^= AES_POLY
        b >>= 1
    return p


def aes_inv(a: int) -> int:
    if a == 0:
        return 0
    r = 1
    for _ in range(254):
        r = aes_mul(r, a)
    return r


def affine(b: int) -> int:
    out = 0
    for i in range(8):
        bit = ((b >> i) ^ (b >> ((i + 4) % 8)) ^ (b >> ((i + 5) % 8)) ^ (b >> ((i + 6) % 8))
               ^ (b >> ((i + 7) % 8)) ^ (0x63 >> i)) & 1
        out |= bit << i
    return out


SBOX = [affine(aes_inv(x)) for x in range(256)]
INV_SBOX = [0] * 256
for _x, _s in enumerate(SBOX):
    INV_SBOX[_s] = _x

# tower elements are ints: GF4 2 bits (W coefficient high), GF16 = (hi GF4 << 2) | lo,
# GF256 = (hi GF16 << 4) | lo


def g4_mul(a, b):
    a1, a0, b1, b0 = a >> 1, a & 1, b >> 1, b & 1
    hi = (a1 & b1) ^ (a1 & b0) ^ (a0 & b1)
    lo = (a1 & b1) ^ (a0 & b0)
    return (hi << 1) | lo


MU = 2  # W; set by configure()
LAM = 0  # set by configure()


def g16_mul(a, b):
    a1, a0, b1, b0 = a >> 2, a & 3, b >> 2, b & 3
    hi = g4_mul(a1, b1) ^ g4_mul(a1, b0) ^ g4_mul(a0, b1)
    lo = g4_mul(g4_mul(a1, b1), MU) ^ g4_mul(a0, b0)
    return (hi << 2) | lo


def lambdas():
    """The lam making Y^2 + Y + lam irreducible over the current GF(16)."""
    squares_plus = {g16_mul(y, y) ^ y for y in range(16)}
    return [lam for lam in range(1, 16) if lam not in squares_plus]


def configure(mu: int, lam: int) -> None:
    global MU, LAM
    if mu not in (2, 3):
        raise ValueError("mu must be W (2) or W^2 (3)")
    MU = mu
    if lam not in lambdas():
        raise ValueError(f"Y^2 + Y + {lam:#x} is reducible")
    LAM = lam


def g256_mul(a, b):
    ah, al, bh, bl = a >> 4, a & 15, b >> 4, b & 15
    hi = g16_mul(ah, bh) ^ g16_mul(ah, bl) ^ g16_mul(al, bh)
    lo = g16_mul(g16_mul(ah, bh), LAM) ^ g16_mul(al, bl)
    return (hi << 4) | lo


def g256_pow(a, e):
    r = 1
    for _ in range(e):
        r = g256_mul(r, a)
    return r


def roots():
    """Roots of the AES polynomial in the current tower field."""
    return [b for b in range(2, 256)
            if g256_pow(b, 8) ^ g256_pow(b, 4) ^ g256_pow(b, 3) ^ b ^ 1 == 0]


def isomorphism(beta: int):
    """8x8 matrix T (list of 8 column ints) with T(x^i) = beta^i, checked to
    be a bijection and multiplicative."""
    if beta not in roots():
        raise ValueError(f"{beta:#x} is not a root of the AES polynomial")
    cols = [g256_pow(beta, i) for i in range(8)]

    def T(x):
        return mat_apply(cols, x)

    if len({T(x) for x in range(256)}) != 256:
        raise ValueError("not a bijection")
    if not all(T(aes_mul(a, b)) == g256_mul(T(a), T(b)) for a in range(0, 256, 3) for b in range(0, 256, 7)):
        raise ValueError("not multiplicative")
    return cols, T


def mat_apply(cols, x):
    r = 0
    for i in range(8):
        if (x >> i) & 1:
            r ^= cols[i]
    return r


def mat_from_fn(fn):
    return [fn(1 << i) for i in range(8)]


def mat_inverse(cols):
    table = {mat_apply(cols, x): x for x in range(256)}
    return [table[1 << i] for i in range(8)]


# --------------------------------------------------------------- circuit ----

class Circuit:
    """Signals are frozensets of atom ids (XOR of atoms).  Atoms 0..7 are the
    input slices (99 = all-ones when a constant is needed); AND gates create
    new atoms.  Building only records the AND gates and outputs; `finish`
    then emits the XOR networks layer by layer (AND depth), each layer's
    operand combinations built as one short linear program (see _reduce),
    starting from the atoms and every earlier XOR node in their span."""

    def __init__(self, prefix="t"):
        self.prefix = prefix
        self.atoms = {i: f"x{i}" for i in range(8)}
        self.depth = {i: 0 for i in range(8)}
        self.gates = []  # (atom, opA set, opB set)
        self.lines = []
        self.ops = []
        self.n = 0
        self.n_and = 0
        self.n_xor = 0

    def AND(self, a: frozenset, b: frozenset) -> frozenset:
        if not a or not b:
            raise ValueError("AND with a zero signal")
        atom = 1000 + len(self.gates)
        d = 1 + max(self.depth[x] for x in (a | b))
        self.depth[atom] = d
        self.gates.append((atom, a, b))
        return frozenset([atom])

    def _new(self):
        name = f"{self.prefix}{self.n}"
        self.n += 1
        return name

    def _xor(self, u: str, v: str) -> str:
        name = self._new()
        self.lines.append(f"const W {name} = {u} ^ {v};")
        self.ops.append((name, "^", u, v))
        self.n_xor += 1
        return name

    def _reduce(self, targets):
        """Build every target (set of atoms) with few XORs; returns {target: name}.

        Signals are vectors over the targets' atoms (bit i = atom i of the
        sorted support).  The base starts as those atoms plus every signal
        already built inside their span.  ell[v] is the least number of base
        signals summing to v, for every v of the span; adding s to the base
        gives ell'[v] = min(ell[v], 1 + ell[v ^ s]) exactly (s is used at
        most once).  Each step adds the pair sum that is itself a target, or
        else the one giving the smallest total of ell over the targets (ties:
        the largest sum of squares, so that near targets finish first)."""
        todo = [t for t in targets if t not in self.built]
        if todo:
            support = sorted(set().union(*todo))
            idx = {a: i for i, a in enumerate(support)}
            span = set(support)

            def vec(sig):
                return sum(1 << idx[a] for a in sig)

            base = {1 << idx[a]: self.atoms[a] for a in support}
            for sig, name in self.built.items():
                if len(sig) > 1 and sig <= span:
                    base.setdefault(vec(sig), name)
            every = np.arange(1 << len(support), dtype=np.int64)
            ell = np.full(every.size, 1 << 14, dtype=np.int32)
            ell[0] = 0
            for b in base:
                ell = np.minimum(ell, ell[every ^ b] + 1)
            F = np.array(sorted({vec(t) for t in todo}), dtype=np.int64)
            while (ell[F] > 1).any():
                B = np.array(list(base), dtype=np.int64)
                ii, jj = np.triu_indices(B.size, 1)
                S = B[ii] ^ B[jj]
                fresh = np.array([v not in base for v in S.tolist()])
                S, ii, jj = S[fresh], ii[fresh], jj[fresh]
                new = np.minimum(ell[F][:, None], 1 + ell[F[:, None] ^ S[None, :]])
                is_target = (S[None, :] == F[:, None]).any(axis=0)
                total = new.sum(axis=0) - (1 << 20) * is_target
                c = np.lexsort((-(new.astype(np.int64) ** 2).sum(axis=0), total))[0]
                s = int(S[c])
                base[s] = self._xor(base[int(B[ii[c]])], base[int(B[jj[c]])])
                ell = np.minimum(ell, ell[every ^ s] + 1)
            for t in todo:
                self.built[t] = base[vec(t)]
        return {t: self.built[t] for t in targets}

    def finish(self, outputs):
        self.built = {frozenset([i]): f"x{i}" for i in range(8)}
        if 99 in self.atoms:
            self.built[frozenset([99])] = "ONES"
        levels = sorted({self.depth[g[0]] for g in self.gates})
        for lv in levels:
            gs = [g for g in self.gates if self.depth[g[0]] == lv]
            names = self._reduce({x for g in gs for x in (g[1], g[2])})
            for atom, a, b in gs:
                name = self._new()
                self.lines.append(f"const W {name} = {names[a]} & {names[b]};")
                self.ops.append((name, "&", names[a], names[b]))
                self.n_and += 1
                self.atoms[atom] = name
                self.built[frozenset([atom])] = name
        names = self._reduce(set(outputs))
        return [names[o] for o in outputs]


def X(*sigs) -> frozenset:
    r = frozenset()
    for s in sigs:
        r = r ^ s
    return r


# symbolic tower arithmetic: GF4 = (hi, lo) signals, GF16 = (GF4 hi, GF4 lo), GF256 = (GF16, GF16)

def s4_mul(c, a, b):
    (a1, a0), (b1, b0) = a, b
    p = c.AND(a1, b1)
    q = c.AND(a0, b0)
    r = c.AND(X(a1, a0), X(b1, b0))
    return (X(r, q), X(p, q))


def s4_scale_mu(a):  # times mu: W (a1 W + a0) = (a1 + a0) W + a1;  W^2 (a1 W + a0) = a0 W + (a1 + a0)
    a1, a0 = a
    return (X(a1, a0), a1) if MU == 2 else (a0, X(a1, a0))


def s4_sq(a):  # squaring (= inversion in GF(4))
    a1, a0 = a
    return (a1, X(a1, a0))


def s4_add(a, b):
    return (X(a[0], b[0]), X(a[1], b[1]))


def s16_mul(c, a, b):
    (A1, A0), (B1, B0) = a, b
    P = s4_mul(c, A1, B1)
    Q = s4_mul(c, A0, B0)
    R = s4_mul(c, s4_add(A1, A0), s4_add(B1, B0))
    return (s4_add(R, Q), s4_add(s4_scale_mu(P), Q))


def s16_add(a, b):
    return (s4_add(a[0], b[0]), s4_add(a[1], b[1]))


def s16_inv(c, a):
    A1, A0 = a
    e = s4_add(s4_add(s4_scale_mu(s4_sq(A1)), s4_mul(c, A1, A0)), s4_sq(A0))
    e = s4_sq(e)  # inverse in GF(4)
    return (s4_mul(c, A1, e), s4_mul(c, s4_add(A1, A0), e))


def s16_linear(a, fn):
    """Apply a GF(2)-linear map on GF(16) (given on ints) to a signal quadruple."""
    bits = [a[1][1], a[1][0], a[0][1], a[0][0]]  # bit0 .. bit3
    out = []
    for j in range(4):
        acc = frozenset()
        for i in range(4):
            if (fn(1 << i) >> j) & 1:
                acc = acc ^ bits[i]
        out.append(acc)
    return ((out[3], out[2]), (out[1], out[0]))


def s256_inv(c, x):
    H, L = x
    t = s16_add(s16_add(s16_linear(H, lambda v: g16_mul(g16_mul(v, v), LAM)), s16_mul(c, H, L)),
                s16_linear(L, lambda v: g16_mul(v, v)))
    d = s16_inv(c, t)
    return (s16_mul(c, H, d), s16_mul(c, s16_add(H, L), d))


def bits_to_tower(sigs):
    """8 bit-signals (bit 0 first) -> tower structure."""
    b = sigs
    return (((b[7], b[6]), (b[5], b[4])), ((b[3], b[2]), (b[1], b[0])))


def tower_to_bits(t):
    ((h1, h0), (l1, l0)) = t[0], t[1]
    return [l0[1], l0[0], l1[1], l1[0], h0[1], h0[0], h1[1], h1[0]]


def linear_on_sigs(sigs, cols):
    """y = M x for a matrix given by columns; sigs are the 8 signals of x."""
    out = []
    for j in range(8):
        acc = frozenset()
        for i in range(8):
            if (cols[i] >> j) & 1:
                acc = acc ^ sigs[i]
        out.append(acc)
    return out


# (mu, lam, beta) per direction: the fewest gates found by search()
PARAMS = {False: (2, 0xA, 0x68), True: (2, 0xC, 0x42)}


def build(inverse: bool, params=None):
    mu, lam, beta = params if params is not None else PARAMS[inverse]
    configure(mu, lam)
    cols, T = isomorphism(beta)
    Tinv = mat_inverse(cols)
    A = mat_from_fn(lambda v: affine(v) ^ 0x63)  # linear part of the affine map
    Ainv = mat_inverse(A)
    c = Circuit("t")
    xs = [frozenset([i]) for i in range(8)]
    if not inverse:
        top = cols
        bottom = [mat_apply(A, mat_apply(Tinv, 1 << i)) for i in range(8)]
        const = 0x63
        pre_const = 0
    else:
        # S^-1(y) = T^-1 inv(T A^-1 (y + 63)); the constant enters before the linear map:
        # T A^-1 (y + 63) = T A^-1 y + T A^-1 63
        top = [mat_apply(cols, mat_apply(Ainv, 1 << i)) for i in range(8)]
        bottom = Tinv
        const = 0
        pre_const = mat_apply(cols, mat_apply(Ainv, 0x63))
    tin = linear_on_sigs(xs, top)
    # the constant on the inverse path is a NOT on some tower bits: fold it as
    # a "ones" atom handled by complementing the built signal (see NOTS below)
    tower = bits_to_tower(tin)
    inv = s256_inv(c, tower) if pre_const == 0 else None
    if inv is None:
        # add the constant by complementing the affected input combinations:
        # realise with an explicit all-ones atom
        c.atoms[99] = "ONES"
        c.depth[99] = 0
        tin = [s ^ (frozenset([99]) if (pre_const >> j) & 1 else frozenset()) for j, s in enumerate(tin)]
        inv = s256_inv(c, bits_to_tower(tin))
    ibits = tower_to_bits(inv)
    outs = linear_on_sigs(ibits, bottom)
    names = c.finish(outs)
    return c, names, const


def evaluate(c: Circuit, names, const, x: int) -> int:
    env = {f"x{i}": (x >> i) & 1 for i in range(8)}
    env["ONES"] = 1
    for dst, op, a, b in c.ops:
        env[dst] = (env[a] ^ env[b]) if op == "^" else (env[a] & env[b])
    y = 0
    for j, n in enumerate(names):
        y |= env[n] << j
    return y ^ const


def emit(c: Circuit, names, const, fname: str) -> str:
    body = ["  " + ln for ln in c.lines]
    for j, n in enumerate(names):
        neg = "~" if (const >> j) & 1 else ""
        body.append(f"  x{j}_out = {neg}{n};")
    args = ", ".join(f"W& x{j}_out" for j in range(8))
    pre = []
    for j in range(8):
        pre.append(f"  const W x{j} = x{j}_out;")
    uses_ones = any("ONES" in ln for ln in c.lines)
    if uses_ones:
        pre.append("  const W ONES = ~W(0);")
    return (f"// {c.n_and} AND + {c.n_xor} XOR gates (NOTs folded into outputs)\n"
            f"template <class W>\nAESGPU_BS_HD void {fname}({args}) {{\n"
            + "\n".join(pre + body) + "\n}\n")


def check(c: Circuit, names, const, table, what: str) -> None:
    for x in range(256):
        got = evaluate(c, names, const, x)
        if got != table[x]:
            raise SystemExit(f"{what}: circuit wrong at {x}: {got} != {table[x]}")


def search() -> None:
    """Gate counts for every (mu, lam, beta); prints the best per direction."""
    best = {}
    for mu in (2, 3):
        configure(mu, lambdas()[0])
        for lam in lambdas():
            configure(mu, lam)
            for beta in roots():
                for inverse, table in ((False, SBOX), (True, INV_SBOX)):
                    c, names, const = build(inverse, (mu, lam, beta))
                    check(c, names, const, table, f"{(mu, lam, beta)}")
                    gates = c.n_and + c.n_xor
                    print(f"inverse={inverse} mu={mu} lam={lam:#x} beta={beta:#x}: "
                          f"{c.n_and} AND + {c.n_xor} XOR", flush=True)
                    if inverse not in best or gates < best[inverse][0]:
                        best[inverse] = (gates, (mu, lam, beta))
    for inverse in (False, True):
        gates, (mu, lam, beta) = best[inverse]
        print(f"best {'inverse' if inverse else 'forward'}: ({mu}, {lam:#x}, {beta:#x}), {gates} gates")


def main():
    out = []
    params = []
    for inverse, fname, table in ((False, "bs_sbox", SBOX), (True, "bs_inv_sbox", INV_SBOX)):
        c, names, const = build(inverse)
        check(c, names, const, table, fname)
        out.append(emit(c, names, const, fname))
        mu, lam, beta = PARAMS[inverse]
        params.append(f"// {fname}: mu = {'W' if mu == 2 else 'W^2'}, lambda = {lam:#x}, beta = {beta:#x}\n")
        print(f"{fname}: {c.n_and} AND, {c.n_xor} XOR, verified on all 256 inputs")
    header = (
        "// aes_bitslice_circuit.cuh — GENERATED by gen_bitslice.py; do not edit.\n"
        "//\n"
        "// SubBytes and InvSubBytes (FIPS-197 §5.1.1, §5.3.2) as Boolean circuits on\n"
        "// bit-slice words: x{j} holds bit j (bit 0 = least significant) of the byte\n"
        "// being substituted, one independent byte per bit position of W.  Built\n"
        "// from inversion in the tower field GF(((2^2)^2)^2), with XOR layers as\n"
        "// short linear programs (see the generator), checked on all 256 inputs\n"
        "// before emission.  Tower parameters and the root beta that fixes the\n"
        "// isomorphism from the AES basis:\n"
        + "".join(params) +
        "#pragma once\n\n"
        "#if defined(__CUDACC__)\n#define AESGPU_BS_HD __host__ __device__ __forceinline__\n"
        "#else\n#define AESGPU_BS_HD inline\n#endif\n\n"
        "namespace aesgpu {\n\n" + "\n".join(out) + "\n}  // namespace aesgpu\n")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "aes_bitslice_circuit.cuh")
    with open(path, "w") as f:
        f.write(header)
    print(f"wrote {path}")


if __name__ == "__main__":
    if "--search" in sys.argv[1:]:
        search()
    else:
        main()
