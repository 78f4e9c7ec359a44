#!/usr/bin/env python3
"""Generate aes_bitslice_circuit.cuh: the AES S-box and inverse S-box as
straight-line Boolean circuits (AND / XOR / NOT) on bit-slice words.

Route (FIPS-197 §5.1.1 defines SubBytes as inversion in GF(2^8) followed by
an affine map; the inversion is computed here in a tower of fields):

  GF(4)   = GF(2)[W] / (W^2 + W + 1)
  GF(16)  = GF(4)[Z] / (Z^2 + Z + mu),      mu = W
  GF(256) = GF(16)[Y] / (Y^2 + Y + lam),    lam: the first GF(16) constant
                                            making the polynomial irreducible
  inverse of h*Y + l:  d = (h^2*lam + h*l + l^2)^-1,  result (h*d)*Y + (h+l)*d
  inverse in GF(16) the same way over GF(4); inverse in GF(4) = squaring.

An isomorphism T from the AES polynomial basis to the tower basis is found
by searching the tower field for a root of x^8 + x^4 + x^3 + x + 1.  Then
  S(x)    = A . T^-1 . inv(T . x) + 0x63
  S^-1(y) = T^-1 . inv(T . A^-1 . (y + 0x63))
with A the affine matrix.  Every signal is tracked as a set of "atoms"
(input bits and AND outputs) combined by XOR; XOR networks are emitted on
demand with reuse of already-built combinations, and the whole circuit is
evaluated on all 256 inputs before anything is written.

Usage: python gen_bitslice.py   (writes aes_bitslice_circuit.cuh beside itself)
"""
from __future__ import annotations

import os

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


MU = 2  # W


def g16_mul(a, b):
    a1, a0, b1, b0 = a >> 2, a & 3, b >> 2, b & 3
    hi = g4_mul(a1, b1) ^ g4_mul(a1, b0) ^ g4_mul(a0, b1)
    lo = g4_mul(g4_mul(a1, b1), MU) ^ g4_mul(a0, b0)
    return (hi << 2) | lo


def _pick_lambda():
    squares_plus = {g16_mul(y, y) ^ y for y in range(16)}
    for lam in range(1, 16):
        if lam not in squares_plus:
            return lam
    raise RuntimeError("no irreducible Y^2 + Y + lam")


LAM = _pick_lambda()


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


def find_isomorphism():
    """8x8 matrix T (list of 8 column ints) with T(x^i) = beta^i, beta a root
    of the AES polynomial in the tower field, checked to be multiplicative."""
    for beta in range(2, 256):
        # beta^8 + beta^4 + beta^3 + beta + 1 == 0
        v = g256_pow(beta, 8) ^ g256_pow(beta, 4) ^ g256_pow(beta, 3) ^ beta ^ 1
        if v != 0:
            continue
        cols = [g256_pow(beta, i) for i in range(8)]

        def T(x, cols=cols):
            r = 0
            for i in range(8):
                if (x >> i) & 1:
                    r ^= cols[i]
            return r

        if len({T(x) for x in range(256)}) != 256:
            continue
        ok = all(T(aes_mul(a, b)) == g256_mul(T(a), T(b)) for a in range(0, 256, 3) for b in range(0, 256, 7))
        if ok:
            return cols, T
    raise RuntimeError("no isomorphism found")


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
    operand combinations reduced with Paar's greedy common-pair elimination
    and earlier XOR nodes reused where one is contained in a target."""

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
        """Build every target (set of atoms) with few XORs; returns {target: name}."""
        # each working target: set of variable names still to combine
        work = {}
        for t in targets:
            if t in self.built:
                continue
            rem = set(t)
            vars_ = set()
            # reuse the largest earlier XOR nodes contained in the target
            while True:
                best = None
                for k, name in self.built.items():
                    if len(k) > 1 and k <= rem and (best is None or len(k) > len(best[0])):
                        best = (k, name)
                if best is None:
                    break
                rem -= best[0]
                vars_.add(best[1])
            vars_ |= {self.atoms[a] for a in rem}
            work[t] = vars_
        # Paar: repeatedly combine the most frequent pair
        while True:
            counts = {}
            for vs in work.values():
                if len(vs) < 2:
                    continue
                lst = sorted(vs)
                for i in range(len(lst)):
                    for j in range(i + 1, len(lst)):
                        counts[(lst[i], lst[j])] = counts.get((lst[i], lst[j]), 0) + 1
            if not counts:
                break
            pair = max(sorted(counts), key=lambda k: counts[k])
            w = self._xor(*pair)
            for vs in work.values():
                if pair[0] in vs and pair[1] in vs:
                    vs.discard(pair[0])
                    vs.discard(pair[1])
                    vs.add(w)
        for t, vs in work.items():
            (name,) = vs
            self.built[t] = name
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


def s4_scale_mu(a):  # times W
    a1, a0 = a
    return (X(a1, a0), a1)


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


def build(inverse: bool):
    cols, T = find_isomorphism()
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


def main():
    out = []
    for inverse, fname, table in ((False, "bs_sbox", SBOX), (True, "bs_inv_sbox", INV_SBOX)):
        c, names, const = build(inverse)
        for x in range(256):
            got = evaluate(c, names, const, x)
            if got != table[x]:
                raise SystemExit(f"{fname}: circuit wrong at {x}: {got} != {table[x]}")
        out.append(emit(c, names, const, fname))
        print(f"{fname}: {c.n_and} AND, {c.n_xor} XOR, verified on all 256 inputs")
    header = (
        "// aes_bitslice_circuit.cuh — GENERATED by gen_bitslice.py; do not edit.\n"
        "//\n"
        "// SubBytes and InvSubBytes (FIPS-197 §5.1.1, §5.3.2) as Boolean circuits on\n"
        "// bit-slice words: x{j} holds bit j (bit 0 = least significant) of the byte\n"
        "// being substituted, one independent byte per bit position of W.  Built\n"
        f"// from inversion in the tower field GF(((2^2)^2)^2) with mu = W, lambda = {LAM:#x}\n"
        "// (see the generator), checked on all 256 inputs before emission.\n"
        "#pragma once\n\n"
        "#if defined(__CUDACC__)\n#define AESGPU_BS_HD __host__ __device__ __forceinline__\n"
        "#else\n#define AESGPU_BS_HD inline\n#endif\n\n"
        "namespace aesgpu {\n\n" + "\n".join(out) + "\n}  // namespace aesgpu\n")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "aes_bitslice_circuit.cuh")
    with open(path, "w") as f:
        f.write(header)
    print(f"wrote {path}")


if __name__ == "__main__":
    main()
