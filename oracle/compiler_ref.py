"""Reference (oracle) implementation of the paper's compiler-side algorithms.

Test infrastructure only.  Written from the paper's text:

* dependency DAG with commutation used to drop edges (Sec. 3, the DAG
  description below Algorithm 1);
* Algorithm 1, the greedy pass that inserts PermuteQubits instructions
  (Sec. 3), with the readings stated in `alg1`;
* Algorithm 2, the decomposition sigma -> sigma1 -> sigma2 -> sigma'
  (Appendix A);
* the 8.5x communication-overhead time model (Sec. 4, Figs. 2-3 discussion).

Locality rule (Sec. 2 and Appendix C): a gate needs communication iff it acts
non-diagonally on a global qubit -- a global control or a diagonal gate on a
global qubit needs none.  Qubit q is local under sigma iff sigma(q) < m.
"""
from __future__ import annotations

from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

# per-qubit action class: gates of the same class on a shared qubit commute
CLS_Z, CLS_X, CLS_N = 0, 1, 2


def _diag2(m) -> bool:
    m = np.asarray(m).reshape(2, 2)
    return m[0, 1] == 0 and m[1, 0] == 0


def _xtype2(m) -> bool:
    """2x2 that is a function of X: a I + b X."""
    m = np.asarray(m).reshape(2, 2)
    return m[0, 0] == m[1, 1] and m[0, 1] == m[1, 0]


def qubit_classes(g) -> List[int]:
    """Action class of gate g on each of its qubits (same order as g.qubits)."""
    k = g.kind
    if k in ("RZ", "Z", "S", "T", "P"):
        return [CLS_Z]
    if k in ("RX", "X"):
        return [CLS_X]
    if k in ("H", "Y", "RY"):
        return [CLS_N]
    if k == "U1":
        return [CLS_Z if _diag2(g.matrix) else (CLS_X if _xtype2(g.matrix) else CLS_N)]
    if k in ("CZ", "CP"):
        return [CLS_Z, CLS_Z]
    if k == "CNOT":
        return [CLS_Z, CLS_X]
    if k == "CU":
        t = CLS_Z if _diag2(g.matrix) else (CLS_X if _xtype2(g.matrix) else CLS_N)
        return [CLS_Z, t]
    return [CLS_N] * len(g.qubits)   # SWAP, U2, UK: no commutation assumed


def nondiag_qubits(g) -> Tuple[int, ...]:
    """Qubits on which g acts non-diagonally (those that decide locality)."""
    return tuple(q for q, c in zip(g.qubits, qubit_classes(g)) if c != CLS_Z)


def build_dag(gates: Sequence) -> List[List[int]]:
    """Immediate predecessors of every gate.  Gate j depends on an earlier gate
    i iff they share a qubit on which their classes differ (or either is N).
    Per qubit, consecutive gates of one commuting class (Z or X) form a group;
    a gate's predecessors on that qubit are the members of the latest group it
    does not commute with."""
    preds: List[set] = [set() for _ in gates]
    state: Dict[int, Tuple[int, List[int], List[int]]] = {}   # q -> (cls, cur, prev)
    for j, g in enumerate(gates):
        for q, c in zip(g.qubits, qubit_classes(g)):
            cls, cur, prev = state.get(q, (None, [], []))
            if cls is not None and c == cls and c != CLS_N:
                preds[j].update(prev)
                cur = cur + [j]
            else:
                preds[j].update(cur)
                prev, cur, cls = cur, [j], c
            state[q] = (cls, cur, prev)
    return [sorted(p) for p in preds]


def is_local(g, sigma: Sequence[int], m: int) -> bool:
    return all(sigma[q] < m for q in nondiag_qubits(g))


def _swap(sigma: Sequence[int], l: int, g: int) -> List[int]:
    s = list(sigma)
    s[l], s[g] = s[g], s[l]
    return s


def alg1(n: int, m: int, gates: Sequence, scoring: str = "closure",
         max_steps: Optional[int] = None):
    """Algorithm 1 (Sec. 3).  Returns (program, stats); program items are
    ("gate", index, needs_comm) and ("permute", sigma').

    Readings where the pseudo-code is silent or, taken literally, fails:
    * the scheduling sweep visits the remaining vertices in program order;
      removing a vertex exposes its successors later in the same sweep;
    * local / global qubits "according to sigma" are taken in ascending qubit
      order; sigma o (l g) exchanges the storage positions of qubits l and g;
    * scoring="closure" (default): a candidate's score is the number of gates
      the next sweep would schedule under it -- how many gates the exchange
      lets run on local qubits (Sec. 3); the first best candidate
      wins (the strict '>' of the comparison).  With it the pass reproduces
      the ~3.5% of Sec. 4 / Fig. 3;
    * scoring="frontier": the number of frontier gates (no incoming edges) the
      candidate makes local, ties broken by the number of all remaining gates
      it makes local, then by the first candidate;
    * scoring="literal": the count of all remaining gates local under the
      candidate with the threshold 0, exactly as printed; it need not
      terminate, so `max_steps` bounds it and a RuntimeError reports it;
    * the else branch takes the first frontier vertex in program order.
    """
    G = len(gates)
    preds = build_dag(gates)
    succs: List[List[int]] = [[] for _ in range(G)]
    for j, ps in enumerate(preds):
        for i in ps:
            succs[i].append(j)
    npred = np.array([len(p) for p in preds], dtype=np.int64)
    nd = [nondiag_qubits(g) for g in gates]
    done = np.zeros(G, dtype=bool)
    sigma = list(range(n))
    program = []
    remaining = G
    steps = 0
    n_comm = 0
    n_perm = 0

    def schedule(v, comm):
        nonlocal remaining
        done[v] = True
        remaining -= 1
        for s in succs[v]:
            npred[s] -= 1
        program.append(("gate", v, comm))

    def sweep():
        for v in range(G):
            if not done[v] and npred[v] == 0 and all(sigma[q] < m for q in nd[v]):
                schedule(v, False)

    while remaining:
        steps += 1
        if max_steps is not None and steps > max_steps:
            raise RuntimeError("Algorithm 1 did not terminate within max_steps")
        sweep()
        if not remaining:
            break
        loc = [q for q in range(n) if sigma[q] < m]
        glo = [q for q in range(n) if sigma[q] >= m]
        rem = [v for v in range(G) if not done[v]]
        front = [v for v in rem if npred[v] == 0]
        best, best_score = None, None
        if scoring in ("frontier", "literal"):
            prim, sec = _score_counts(rem, front, nd, sigma, m, loc, glo)
            if scoring == "literal":
                prim = sec
                sec = np.zeros_like(sec)
            for li, l in enumerate(loc):
                for gi, g in enumerate(glo):
                    sc = (int(prim[li, gi]), int(sec[li, gi]))
                    if best_score is None or sc > best_score:
                        best, best_score = (l, g), sc
        elif scoring == "closure":
            sc = _closure_counts(rem, preds, nd, done, sigma, m, loc, glo)
            for li, l in enumerate(loc):
                for gi, g in enumerate(glo):
                    s = (int(sc[li, gi]),)
                    if best_score is None or s > best_score:
                        best, best_score = (l, g), s
        else:
            raise ValueError(scoring)
        if best is not None and best_score[0] > 0:
            sigma = _swap(sigma, *best)
            program.append(("permute", list(sigma)))
            n_perm += 1
        else:
            v = front[0]
            schedule(v, True)
            n_comm += 1
    stats = {"n_gates": G, "n_comm_gates": n_comm, "n_permutes": n_perm,
             "comm_fraction": (n_comm + n_perm) / max(G, 1)}
    return program, stats


def _score_counts(rem, front, nd, sigma, m, loc, glo):
    """prim[l,g] = frontier gates local under sigma o (l g);
    sec[l,g] = remaining gates local under sigma o (l g)."""
    li = {q: i for i, q in enumerate(loc)}
    gi = {q: i for i, q in enumerate(glo)}
    prim = np.zeros((len(loc), len(glo)), dtype=np.int64)
    sec = np.zeros((len(loc), len(glo)), dtype=np.int64)
    front_set = set(front)
    for v in rem:
        gl = [q for q in nd[v] if sigma[q] >= m]
        if len(gl) > 1:
            continue
        lmask = np.ones(len(loc), dtype=bool)
        for q in nd[v]:
            if q in li:
                lmask[li[q]] = False      # moving a needed local qubit out breaks it
        if len(gl) == 0:
            sec[lmask, :] += 1
            if v in front_set:
                prim[lmask, :] += 1
        else:
            sec[lmask, gi[gl[0]]] += 1
            if v in front_set:
                prim[lmask, gi[gl[0]]] += 1
    return prim, sec


def _closure_counts(rem, preds, nd, done, sigma, m, loc, glo):
    """Number of gates one program-order sweep schedules under each candidate."""
    C = len(loc) * len(glo)
    cl = np.repeat(np.arange(len(loc)), len(glo))
    cg = np.tile(np.arange(len(glo)), len(loc))
    n = len(sigma)
    # local[c, q] under candidate c
    local = np.zeros((C, n), dtype=bool)
    base = np.array([s < m for s in sigma])
    local[:] = base
    loc_a = np.array(loc)
    glo_a = np.array(glo)
    local[np.arange(C), loc_a[cl]] = False
    local[np.arange(C), glo_a[cg]] = True
    sched: Dict[int, np.ndarray] = {}
    count = np.zeros(C, dtype=np.int64)
    ones = np.ones(C, dtype=bool)
    for v in rem:
        ok = ones.copy()
        for p in preds[v]:
            if not done[p]:
                ok &= sched[p]
        for q in nd[v]:
            ok &= local[:, q]
        sched[v] = ok
        count += ok
    return count.reshape(len(loc), len(glo))


def original_comm_fraction(n: int, m: int, gates: Sequence) -> float:
    """Fraction of gates needing communication when run in program order with
    the identity permutation."""
    ident = list(range(n))
    return sum(0 if is_local(g, ident, m) else 1 for g in gates) / max(len(gates), 1)


def model_time(n_local: float, n_comm: float, overhead: float = 8.5) -> float:
    """The paper's simplified time model: a communicating operation costs
    `overhead` times a local one (Fig. 2 caption)."""
    return n_local + overhead * n_comm


def model_reduction(comm_orig: float, comm_opt: float, overhead: float = 8.5) -> float:
    """1 - t_opt / t_orig with fractions of the original gate count (Sec. 4)."""
    return 1.0 - model_time(1.0 - comm_opt, comm_opt, overhead) / model_time(1.0 - comm_orig, comm_orig, overhead)


def alg2(n: int, m: int, sigma: Sequence[int], sigma_new: Sequence[int]):
    """Algorithm 2 (Appendix A): intermediate permutations sigma1, sigma2 with
    sigma -> sigma1 reordering local qubits among themselves, sigma1 -> sigma2
    reordering global qubits among themselves, sigma2 -> sigma' exchanging
    local/global pairs.  Permutations map qubit -> position; positions not
    assigned by a loop keep the previous step's qubit."""
    inv = [0] * n
    for q in range(n):
        inv[sigma[q]] = q
    inv1 = list(inv)                       # sigma1^{-1}; global positions unchanged
    for p in range(m):
        pp = sigma_new[inv[p]]
        while pp >= m:
            pp = sigma_new[inv[pp]]
        inv1[pp] = inv[p]
    inv2 = list(inv1)                      # sigma2^{-1}; local positions unchanged
    for p in range(m, n):
        pp = sigma_new[inv1[p]]
        while pp < m:
            pp = sigma_new[inv1[pp]]
        inv2[pp] = inv1[p]
    s1 = [0] * n
    s2 = [0] * n
    for p in range(n):
        s1[inv1[p]] = p
        s2[inv2[p]] = p
    return s1, s2
