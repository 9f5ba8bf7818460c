"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of the simulation method itself: it only draws
random numbers and lays out circuits.  Both sides of every parity test take
their gates from here, so neither side generates gates for the other.

Contents
--------
* ``SplitMix64`` counter generator (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014; the finaliser constants are
  the published ones) and Box-Muller normal deviates in FP64.
* Haar-random unitaries by the method of Mezzadri, "How to generate random
  matrices from the classical compact groups", Notices AMS 54 (2007):
  QR of a complex Ginibre matrix, then a phase fix by the diagonal of R.
  The paper draws every gate of its experiments from the Haar measure
  (Fig. 1, Fig. 2 captions).
* Brickwork circuits of nearest-neighbour two-qubit gates (the paper restricts
  itself to linear nearest-neighbour gates, Section "The matrix product
  formalism").  Layer l holds the pairs (0,1),(2,3),... when l is even and
  (1,2),(3,4),... when l is odd.  Gates inside a layer act on disjoint pairs;
  they are emitted left to right on even layers and right to left on odd
  layers (a serpentine sweep, which keeps a single orthogonality centre next
  to the next gate).
* Textbook Kraus operators of the noise models: two-qubit depolarising noise
  and single-qubit amplitude damping.
* Random circuit batches of uneven size.
* A layered variational ansatz: per layer RY then RZ on every qubit, then RZZ on
  the pairs (0,1), (1,2), ..., (n-2,n-1) in that order, with seeded angles.

Index convention for a gate on qubits (q, q+1): a 4x4 matrix acting on the
basis |s_q s_{q+1}> with s_q the more significant bit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "splitmix64",
    "uniforms",
    "normals",
    "haar_unitary",
    "brickwork_pairs",
    "brickwork_circuit",
    "Circuit",
    "depolarizing_2q_kraus",
    "amplitude_damping_kraus",
    "random_batch_specs",
    "count_brickwork_gates",
    "random_canonical_mps",
    "ansatz_params",
    "ansatz_circuit",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """SplitMix64 output for each counter value: mix(seed + (counter+1)*gamma).

    Counter-based form of the SplitMix64 sequence: the i-th output of a
    generator seeded with ``seed`` is ``splitmix64(seed, i)``.
    """
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (
            np.asarray(counters, dtype=np.uint64) + np.uint64(1)) * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniforms(seed: int, start: int, count: int) -> np.ndarray:
    """``count`` doubles in [0, 1) from counters start .. start+count-1 (53-bit)."""
    z = splitmix64(seed, np.arange(start, start + count, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normals(seed: int, start: int, count: int) -> np.ndarray:
    """``count`` standard normal deviates (Box-Muller on pairs of uniforms).

    Uses 2*ceil(count/2) counters starting at ``start``.
    """
    npair = (count + 1) // 2
    u = uniforms(seed, start, 2 * npair)
    u1 = 1.0 - u[0::2]          # in (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    return out[:count]


def haar_unitary(dim: int, seed: int, index: int, special: bool = True) -> np.ndarray:
    """Haar-random ``dim``x``dim`` unitary number ``index`` of stream ``seed``.

    Each index consumes its own block of 2*dim*dim counters, so the gates of a
    circuit do not depend on the order in which they are drawn.  With
    ``special`` the global phase is fixed so that det U = 1 (a global phase is
    physically irrelevant).
    """
    block = 2 * dim * dim
    g = normals(seed, index * block, block).reshape(2, dim, dim)
    z = (g[0] + 1j * g[1]) / math.sqrt(2.0)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    u = q * (d / np.abs(d))[None, :]
    if special:
        det = np.linalg.det(u)
        u = u * np.exp(-1j * np.angle(det) / dim)
    return np.ascontiguousarray(u)


def brickwork_pairs(n_qubits: int, depth: int) -> list[tuple[int, int]]:
    """(layer, q) for every gate of a brickwork circuit, in serpentine order."""
    out = []
    for layer in range(depth):
        qs = list(range(layer % 2, n_qubits - 1, 2))
        if layer % 2 == 1:
            qs.reverse()
        out.extend((layer, q) for q in qs)
    return out


def count_brickwork_gates(n_qubits: int, depth: int) -> int:
    """Number of two-qubit gates of ``brickwork_pairs(n_qubits, depth)``."""
    even = n_qubits // 2
    odd = (n_qubits - 1) // 2
    return ((depth + 1) // 2) * even + (depth // 2) * odd


@dataclass
class Circuit:
    """A list of nearest-neighbour gates.

    ``qs[g]`` is the left qubit of gate g, ``ops[g]`` its 4x4 unitary.
    ``n_2q`` is the number of two-qubit gates (known before the run starts,
    which the target schedule of the method relies on).
    """
    n_qubits: int
    qs: list[int]
    ops: list[np.ndarray]
    layers: list[int] = field(default_factory=list)
    seed: int = 0

    @property
    def n_2q(self) -> int:
        return len(self.qs)

    def gates(self):
        return list(zip(self.qs, self.ops))

    def adjoint(self) -> "Circuit":
        """The inverse circuit: gates in reverse order, each one conjugate-transposed."""
        return Circuit(self.n_qubits, list(reversed(self.qs)),
                       [np.ascontiguousarray(u.conj().T) for u in reversed(self.ops)],
                       list(reversed(self.layers)), self.seed)

    def ops_array(self) -> np.ndarray:
        """All gates as one (n_2q, 4, 4) complex128 array."""
        if not self.ops:
            return np.zeros((0, 4, 4), np.complex128)
        return np.ascontiguousarray(np.stack(self.ops))


def brickwork_circuit(n_qubits: int, depth: int, seed: int) -> Circuit:
    """Haar-random SU(4) brickwork circuit (seeded)."""
    pairs = brickwork_pairs(n_qubits, depth)
    qs, ops, layers = [], [], []
    for g, (layer, q) in enumerate(pairs):
        qs.append(q)
        layers.append(layer)
        ops.append(haar_unitary(4, seed, g))
    return Circuit(n_qubits, qs, ops, layers, seed)


_PAULI = [
    np.array([[1, 0], [0, 1]], np.complex128),
    np.array([[0, 1], [1, 0]], np.complex128),
    np.array([[0, -1j], [1j, 0]], np.complex128),
    np.array([[1, 0], [0, -1]], np.complex128),
]


def depolarizing_2q_kraus(p: float) -> list[np.ndarray]:
    """Kraus operators of E(rho) = (1-p) rho + p/15 sum_{P != II} P rho P^dagger."""
    ks = [math.sqrt(1.0 - p) * np.eye(4, dtype=np.complex128)]
    for a in range(4):
        for b in range(4):
            if a == 0 and b == 0:
                continue
            ks.append(math.sqrt(p / 15.0) * np.kron(_PAULI[a], _PAULI[b]))
    return ks


def amplitude_damping_kraus(gamma: float) -> list[np.ndarray]:
    """Kraus operators K0 = diag(1, sqrt(1-gamma)), K1 = sqrt(gamma)|0><1|."""
    k0 = np.array([[1.0, 0.0], [0.0, math.sqrt(1.0 - gamma)]], np.complex128)
    k1 = np.array([[0.0, math.sqrt(gamma)], [0.0, 0.0]], np.complex128)
    return [k0, k1]


def random_batch_specs(count: int, seed: int, n_range=(20, 80), depth_range=(10, 30),
                       f_choices=(0.9, 0.99)) -> list[dict]:
    """Sizes of a batch of independent circuits: N, depth, F_min, circuit seed."""
    u = uniforms(seed, 0, 3 * count).reshape(count, 3)
    specs = []
    for i in range(count):
        n = n_range[0] + int(u[i, 0] * (n_range[1] - n_range[0] + 1))
        d = depth_range[0] + int(u[i, 1] * (depth_range[1] - depth_range[0] + 1))
        f = f_choices[int(u[i, 2] * len(f_choices))]
        specs.append({"n_qubits": n, "depth": d, "f_min": f, "seed": seed * 1000 + i + 1})
    return specs


def random_canonical_mps(n, chi_cap, centre, seed, d=2, round_c64=True):
    """Random MPS in canonical form around ``centre`` (synthetic input state).

    Sites left of the centre are random left isometries, sites right of it
    random right isometries (both from the QR of complex Ginibre matrices),
    the centre a random unit tensor; bonds are min(chi_cap, d^min(b, n-b)).
    With ``round_c64`` every entry is first rounded to complex64, so that a
    complex64 copy holds exactly the same numbers.  Returns (sites, bonds).
    """
    bonds = [1] + [min(chi_cap, d ** min(b, n - b)) for b in range(1, n)] + [1]
    sites = []
    off = 0
    for i in range(n):
        cl, cr = bonds[i], bonds[i + 1]
        cnt = cl * d * cr
        g = normals(seed, off, 2 * cnt).reshape(2, cnt)
        off += 2 * cnt + 2
        t = (g[0] + 1j * g[1]).reshape(cl, d, cr)
        if i < centre:
            q, _ = np.linalg.qr(t.reshape(cl * d, cr))
            t = q.reshape(cl, d, cr)
        elif i > centre:
            q, _ = np.linalg.qr(t.reshape(cl, d * cr).conj().T)
            t = q.conj().T.reshape(cl, d, cr)
        else:
            t = t / np.linalg.norm(t)
        if round_c64:
            t = t.astype(np.complex64).astype(np.complex128)
        sites.append(np.ascontiguousarray(t))
    return sites, bonds


def ansatz_params(n_qubits: int, layers: int, seed: int) -> np.ndarray:
    """Seeded angles U[0, 2 pi) of ansatz_circuit: per layer n RY, n RZ, n-1 RZZ angles."""
    return 2.0 * math.pi * uniforms(seed, 0, layers * (3 * n_qubits - 1))


def _ry(t: float) -> np.ndarray:
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], np.complex128)


def _rz(t: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * t), np.exp(0.5j * t)])


def _rzz(t: float) -> np.ndarray:
    a, b = np.exp(-0.5j * t), np.exp(0.5j * t)
    return np.diag([a, b, b, a])


def ansatz_circuit(n_qubits: int, layers: int, params) -> Circuit:
    """The layered ansatz as nearest-neighbour two-qubit gates only.

    Layer l applies RY(a) then RZ(b) to every qubit, then RZZ(g) = exp(-i g Z x Z / 2) to
    (0,1), (1,2), ..., (n-2,n-1) in that order.  Each qubit's single-qubit rotation is folded
    into the first two-qubit gate that touches it: gate (0,1) = RZZ (R_0 x R_1), gate (i,i+1) =
    RZZ (1 x R_{i+1}) for i >= 1, with R = RZ(b) RY(a).  Every angle is exp(-i t P / 2) for a
    Pauli product P, so the parameter-shift rule applies to each.
    """
    p = np.asarray(params, dtype=np.float64).reshape(layers, 3 * n_qubits - 1)
    qs, ops, lay = [], [], []
    eye = np.eye(2, dtype=np.complex128)
    for l in range(layers):
        ry, rz, zz = p[l, :n_qubits], p[l, n_qubits:2 * n_qubits], p[l, 2 * n_qubits:]
        r = [_rz(rz[i]) @ _ry(ry[i]) for i in range(n_qubits)]
        for i in range(n_qubits - 1):
            local = np.kron(r[0], r[1]) if i == 0 else np.kron(eye, r[i + 1])
            qs.append(i)
            ops.append(_rzz(zz[i]) @ local)
            lay.append(l)
    return Circuit(n_qubits, qs, ops, lay, 0)
