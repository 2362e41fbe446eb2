#!/usr/bin/env python3
"""Generate os_generated.cuh: straight-line Obara-Saika code per shell-pair class.

For each class (l_a, l_b) with l_a >= l_b, l <= 2 this emits

  * ``vrr``: one primitive pair's vertical recursion (App. A, Eq. vrr) from the
    scaled seeds S_n = pref * F_n(T), n = 0..L, L = l_a + l_b, adding every
    Theta^0_e with l_a <= |e| <= L into the contracted accumulator ``acc``;
  * ``hrr``: the horizontal recursion (App. A, Eq. hrr) from the contracted
    accumulator to the target block Xi_{ab};

as straight-line code on named registers, templated on the arithmetic type
(double for the FP64 path, float for the FP32 pairs of the mixed form).  Only the intermediates that
some target needs are emitted (a dependency walk from the targets, in the
spirit of the paper's pre-order traversal), and the direction of each step
is chosen to avoid the third VRR term where possible.  The generator also
counts the FP64 operations it emits (FMA = 2 flops), which the library
reports as the algorithmic work of the integral kernel.

Run:  python gen_os.py > os_generated.cuh
"""
from __future__ import annotations

import sys

CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]


def ncart(l):
    return (l + 1) * (l + 2) // 2


def carts(l):
    return [(ax, ay, l - ax - ay) for ax in range(l, -1, -1) for ay in range(l - ax, -1, -1)]


def name_e(e):
    return f"{e[0]}{e[1]}{e[2]}"


class Counter:
    def __init__(self):
        self.fma = self.mul = self.add = 0

    @property
    def flops(self):
        return 2 * self.fma + self.mul + self.add

    @property
    def ops(self):
        return self.fma + self.mul + self.add


def vrr_direction(e):
    """Direction q of the step e - 1_q: the smallest positive component, so
    that the a_q term of Eq. (vrr) drops out whenever some e_q == 1."""
    best = None
    for q in range(3):
        if e[q] > 0 and (best is None or e[q] < e[best]):
            best = q
    return best


def gen_vrr(la, lb):
    L = la + lb
    targets = [(e, 0) for l in range(la, L + 1) for e in carts(l)]
    need = set()
    stack = list(targets)
    while stack:
        node = stack.pop()
        if node in need:
            continue
        need.add(node)
        e, n = node
        if sum(e) == 0:
            continue
        q = vrr_direction(e)
        m = list(e)
        m[q] -= 1
        m = tuple(m)
        stack += [(m, n), (m, n + 1)]
        if m[q] > 0:
            mm = list(m)
            mm[q] -= 1
            mm = tuple(mm)
            stack += [(mm, n), (mm, n + 1)]
    c = Counter()
    lines = []
    diffs = {}
    order = sorted(need, key=lambda x: (sum(x[0]), -x[0][0], -x[0][1], x[1]))
    for (e, n) in order:
        v = f"t{name_e(e)}_{n}"
        if sum(e) == 0:
            lines.append(f"const R {v} = S[{n}];")
            continue
        q = vrr_direction(e)
        Q = "xyz"[q]
        m = list(e)
        m[q] -= 1
        m = tuple(m)
        base = f"fma(PA{Q}, t{name_e(m)}_{n}, -PC{Q} * t{name_e(m)}_{n + 1})"
        c.mul += 1
        c.fma += 1
        if m[q] > 0:
            mm = list(m)
            mm[q] -= 1
            mm = tuple(mm)
            key = (mm, n)
            if key not in diffs:
                dname = f"d{name_e(mm)}_{n}"
                diffs[key] = dname
                lines.append(f"const R {dname} = t{name_e(mm)}_{n} - t{name_e(mm)}_{n + 1};")
                c.add += 1
            lines.append(f"const R {v} = fma(k{m[q]}, {diffs[key]}, {base});")
            c.fma += 1
        else:
            lines.append(f"const R {v} = {base};")
    acc_index = {}
    for (e, _) in targets:
        acc_index[e] = len(acc_index)
        lines.append(f"acc[{acc_index[e]}] += t{name_e(e)}_0;")
        c.add += 1
    kmax = max([0] + [e[vrr_direction(e)] - 1 for (e, n) in need if sum(e) > 0])
    return lines, c, acc_index, kmax


def gen_hrr(la, lb, acc_index, rule):
    L = la + lb
    targets = [(a, b) for a in carts(la) for b in carts(lb)]
    need = set()
    stack = list(targets)

    def step(f):
        qs = [q for q in range(3) if f[q] > 0]
        return qs[0] if rule == 0 else qs[-1]

    while stack:
        node = stack.pop()
        if node in need:
            continue
        need.add(node)
        e, f = node
        if sum(f) == 0:
            continue
        q = step(f)
        g = list(f)
        g[q] -= 1
        g = tuple(g)
        e1 = list(e)
        e1[q] += 1
        e1 = tuple(e1)
        stack += [(e1, g), (e, g)]
    c = Counter()
    lines = []
    order = sorted(need, key=lambda x: (sum(x[1]), -sum(x[0]), x))
    for (e, f) in order:
        v = f"x{name_e(e)}_{name_e(f)}"
        if sum(f) == 0:
            lines.append(f"const R {v} = acc[{acc_index[e]}];")
            continue
        q = step(f)
        Q = "xyz"[q]
        g = list(f)
        g[q] -= 1
        g = tuple(g)
        e1 = list(e)
        e1[q] += 1
        e1 = tuple(e1)
        lines.append(f"const R {v} = fma(AB{Q}, x{name_e(e)}_{name_e(g)}, x{name_e(e1)}_{name_e(g)});")
        c.fma += 1
    for i, a in enumerate(carts(la)):
        for j, b in enumerate(carts(lb)):
            lines.append(f"xi[{i * ncart(lb) + j}] = x{name_e(a)}_{name_e(b)};")
    return lines, c


def main(out=sys.stdout):
    w = out.write
    w("// Generated by gen_os.py -- do not edit.\n")
    w("// Straight-line Obara-Saika VRR (App. A, Eq. vrr) and HRR (Eq. hrr) for the\n")
    w("// 3c-CP integrals of one shell-pair class, with the FP64 operation counts.\n")
    w("#pragma once\n\nnamespace snk {\n\n")
    w("template <int LA, int LB> struct OsClass;\n\n")
    for (la, lb) in CLASSES:
        vl, vc, acc_index, kmax = gen_vrr(la, lb)
        best = None
        for rule in (0, 1):
            hl, hc = gen_hrr(la, lb, acc_index, rule)
            if best is None or hc.ops < best[1].ops:
                best = (hl, hc)
        hl, hc = best
        L = la + lb
        nacc = len(acc_index)
        w(f"// class ({la},{lb}): {len(vl)} VRR statements, VRR {vc.flops} flops per primitive pair,\n")
        w(f"// HRR {hc.flops} flops per contracted pair\n")
        w(f"template <> struct OsClass<{la}, {lb}> {{\n")
        w(f"  static constexpr int L = {L};\n")
        w(f"  static constexpr int NACC = {nacc};\n")
        w(f"  static constexpr int NA = {ncart(la)};\n")
        w(f"  static constexpr int NB = {ncart(lb)};\n")
        w(f"  static constexpr int KMAX = {kmax};\n")
        w(f"  static constexpr int VRR_FLOPS = {vc.flops};\n")
        w(f"  static constexpr int VRR_OPS = {vc.ops};\n")
        w(f"  static constexpr int HRR_FLOPS = {hc.flops};\n")
        w(f"  static constexpr int HRR_OPS = {hc.ops};\n")
        w("  template <typename R>\n")
        w("  __device__ static __forceinline__ void vrr(const R* S, R PAx, R PAy, R PAz, R PCx, R PCy, R PCz,\n")
        w("                                             R k1, R k2, R k3, R* acc) {\n")
        w("    (void)PAx; (void)PAy; (void)PAz; (void)PCx; (void)PCy; (void)PCz; (void)k1; (void)k2; (void)k3;\n")
        for s in vl:
            w("    " + s + "\n")
        w("  }\n")
        w("  template <typename R>\n")
        w("  __device__ static __forceinline__ void hrr(const R* acc, R ABx, R ABy, R ABz, R* xi) {\n")
        w("    (void)ABx; (void)ABy; (void)ABz;\n")
        for s in hl:
            w("    " + s + "\n")
        w("  }\n};\n\n")
    w("}  // namespace snk\n")


if __name__ == "__main__":
    main()
