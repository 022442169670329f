"""Bytecode integrands (the generator's program files for the interpreter
kernels), checked on the CPU: every program is well formed, and a plain
numpy interpretation of it reproduces the oracle's subtracted integrand
(Sec. 2) at two, three and four loops.  At four loops the reference values
are the oracle's, stored by tests/golden/make_four_loop.py at the Eq. (1)
points of fixed Philox counters.

Instruction (64 bits): lo = A | B << 13, hi = XA | ZO << 1 | SPEC << 2 |
NOCOMP << 5 | D << 6; operand >= 4096 selects a constant.  Unless NOCOMP:
X = XA ? A : acc, O = XA ? acc : A, acc = X * B + (ZO ? O : 0); then SPEC
(1 RCP, 2 ABS, 3 ACCW: W += |A| e(B), 4 END); then D != 0 stores acc."""
import struct
from pathlib import Path

import numpy as np
import pytest

from oracle.graphs import enumerate_graphs as o_enum
from oracle.integrand import Integrand

ROOT = Path(__file__).resolve().parents[1]
GEN = ROOT / "paper_1905_08007_b300" / "csrc" / "_gen"
GOLDEN4 = ROOT / "tests" / "golden" / "four_loop_points.txt"


def read_programs(path):
    data = path.read_bytes()
    if path.suffix == ".z":
        import zlib
        data = zlib.decompress(data)
    assert data[:8] == b"QEDVM004"
    (count,) = struct.unpack_from("<I", data, 8)
    off = 16
    progs = {}
    for _ in range(count):
        name = data[off:off + 64].split(b"\0")[0].decode()
        n_lines, n_regs, n_ins, n_kon = struct.unpack_from("<4i", data, off + 64)
        (flops,) = struct.unpack_from("<d", data, off + 80)
        off += 88
        ins = np.frombuffer(data, dtype="<u8", count=n_ins, offset=off)
        off += 8 * n_ins
        kon = np.frombuffer(data, dtype="<f8", count=n_kon, offset=off)
        off += 8 * n_kon
        progs[name] = dict(n_lines=n_lines, n_regs=n_regs, ins=ins, kon=kon, flops=flops)
    assert off == len(data)
    return progs


def interpret(p, z, dtype=np.float64):
    """The fused accumulator / register machine, vectorised over points."""
    z = np.asarray(z, dtype=dtype)
    B, N = z.shape
    R = np.zeros((p["n_regs"], B), dtype=dtype)
    E = np.zeros((p["n_regs"], B), dtype=dtype)
    R[:N] = z.T
    E[:N] = np.abs(z.T)
    K = p["kon"].astype(dtype)
    acc = np.zeros(B, dtype=dtype)
    ae = np.zeros(B, dtype=dtype)
    W = np.zeros(B, dtype=dtype)

    def get(x):
        if x >= 4096:
            return np.full(B, K[x - 4096], dtype=dtype), np.full(B, abs(K[x - 4096]), dtype=dtype)
        return R[x], E[x]

    for w in p["ins"].tolist():
        lo, hi = w & 0xFFFFFFFF, w >> 32
        a, b, d = lo & 8191, (lo >> 13) & 8191, (hi >> 6) & 1023
        xa, zo, spec, nocomp = hi & 1, (hi >> 1) & 1, (hi >> 2) & 7, (hi >> 5) & 1
        (va, ea), (vb, eb) = get(a), get(b)
        if not nocomp:
            X, eX = (va, ea) if xa else (acc, ae)
            O, eO = (acc, ae) if xa else (va, ea)
            Z, eZ = (O, eO) if zo else (0, 0)
            acc, ae = X * vb + Z, eX * eb + eZ
        if spec == 1:
            acc = 1 / acc
            ae = np.abs(acc)
        elif spec == 2:
            ae = np.abs(acc)
        elif spec == 3:
            W = W + np.abs(va) * eb
        elif spec == 4:
            return acc, W
        elif spec != 0:
            raise AssertionError(f"bad special {spec}")
        if d:
            R[d] = acc
            E[d] = ae
    raise AssertionError("program without END")


def _name(g):
    return f"n{g.n}_e{g.e}" + "".join(f"_{s}{t}" for s, t in g.pairs)


def _programs(n):
    path = GEN / f"vm_n{n}.bin.z"
    if not path.exists():
        pytest.skip(f"{path.name} not built")
    return read_programs(path)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_programs_well_formed(n):
    progs = _programs(n)
    if n == 5:
        # the five-loop workload: the graphs five_loop_subset.txt lists
        from paper_1905_08007_b300.five_loop_subset import read
        every = o_enum(5)
        red = [every[i] for i in read()]
    else:
        red = [g for g in o_enum(n) if tuple(g.key()) <= tuple(g.mirror().key())]
    if n == 5:
        # five-loop programs are generated graph by graph on request: a
        # file may hold part of the workload, in its order
        names = [_name(g) for g in red]
        assert progs and set(progs) <= set(names)
    else:
        assert sorted(progs) == sorted(_name(g) for g in red)
    for name, p in progs.items():
        assert p["n_lines"] == 3 * n and p["n_lines"] <= p["n_regs"] <= 1023 and len(p["kon"]) <= 4096
        ins = p["ins"]
        lo, hi = ins & 0xFFFFFFFF, ins >> 32
        a, b, d = lo & 8191, (lo >> 13) & 8191, (hi >> 6) & 1023
        spec = (hi >> 2) & 7
        assert (lo >> 26).max() == 0 and (hi >> 16).max() == 0 and spec.max() <= 4
        end = int(np.argmax(spec == 4))
        assert spec[end] == 4
        ok = lambda x: np.where(x >= 4096, x - 4096 < len(p["kon"]), x < p["n_regs"])   # noqa: E731
        assert ok(a[:end + 1]).all() and ok(b[:end + 1]).all(), name
        st = d[:end + 1][d[:end + 1] != 0]
        assert ((st >= p["n_lines"]) & (st < p["n_regs"])).all(), name
        # END last; no instruction reads the register the previous one writes
        assert end == len(ins) - 1, name
        prev = d[:-1]
        assert not np.any((prev != 0) & ((a[1:] == prev) | (b[1:] == prev))), name


@pytest.mark.parametrize("n,sel", [(2, None), (3, [0, 9, 19, 27])])
def test_programs_match_oracle(n, sel):
    progs = _programs(n)
    red = [(i, g) for i, g in enumerate(o_enum(n)) if tuple(g.key()) <= tuple(g.mirror().key())]
    if sel is not None:
        red = [red[i] for i in sel]
    rng = np.random.default_rng(7)
    for i, g in red:
        z = rng.random((6, g.n_lines)) ** 3 + 1e-3
        z /= z.max(axis=1, keepdims=True)
        fo = Integrand(g)(z, dtype=np.longdouble)
        fv, W = interpret(progs[_name(g)], z, np.longdouble)
        # both sides long double in different operation orders: each within
        # a few ulp(long double) times kappa = sum|monomials| / |f| (W / |f|)
        kappa = (W / np.abs(fv)).astype(float)
        rel = np.abs((fv - fo) / fo).astype(float)
        assert np.all(rel <= 1e-12 + 16 * 2.0 ** -64 * kappa), (_name(g), rel, kappa)
        # the absolute sum bounds the value
        assert np.all(W >= np.abs(fv) * (1 - 1e-12))


def test_four_loop_programs_match_stored_oracle():
    progs = _programs(4)
    if not GOLDEN4.exists():
        pytest.skip("four_loop_points.txt not written")
    rows = [ln.split() for ln in GOLDEN4.read_text().splitlines() if ln and not ln.startswith("#")]
    gs = o_enum(4)
    byg = {}
    for r in rows:
        byg.setdefault(int(r[0]), []).append(r)
    assert len(byg) >= 4
    # every stored graph while there are few (a numpy interpretation of a
    # four-loop program takes a fraction of a second per graph), else the two
    # thirds the GPU test leaves out
    items = sorted(byg.items())
    for gi, rs in (items if len(items) <= 16 else [it for k, it in enumerate(items) if k % 3]):
        z = np.array([[float(v) for v in r[3:15]] for r in rs])
        fo = np.array([np.longdouble(r[15]) for r in rs])
        fv, W = interpret(progs[_name(gs[gi])], z, np.longdouble)
        # both sides are long double in different operation orders: each is
        # within some ulp(long double) times the condition number
        # kappa = (sum of |monomials|) / |f| that the program's W measures;
        # the oracle's explicit 4x4 Dirac algebra cancels more than the
        # expanded polynomials (up to 23 ulp x kappa over the stored points)
        kappa = (W / np.abs(fv)).astype(float)
        rel = np.abs((fv - fo) / fo).astype(float)
        assert np.all(rel <= 1e-12 + 64 * 2.0 ** -64 * kappa), (gi, rel, kappa)


def test_five_loop_programs_match_stored_oracle():
    """The generator's five-loop programs in long double against the
    oracle's stored five-loop values (tests/golden/five_loop_points.txt,
    float64), for the stored graphs whose programs were generated
    (five-loop programs are built on request): within 1e-12 plus 16 x 2^-53
    x kappa where the integrand is well conditioned (kappa = sum of
    |monomials| / |f| <= 1e4).  At strongly cancelling points the float64
    oracle has lost the digits (its explicit Dirac algebra cancels more than
    the generated polynomials), so those points are not compared."""
    path = GEN / "vm_n5.bin.z"
    golden5 = ROOT / "tests" / "golden" / "five_loop_points.txt"
    if not path.exists() or not golden5.exists():
        pytest.skip("five-loop programs or stored points missing")
    progs = read_programs(path)
    gs = o_enum(5)
    byg = {}
    for ln in golden5.read_text().splitlines():
        if ln and not ln.startswith("#"):
            r = ln.split()
            byg.setdefault(int(r[0]), []).append(r)
    n = 0
    for gi, rs in sorted(byg.items()):
        p = progs.get(_name(gs[gi]))
        if p is None:
            continue
        z = np.array([[float(v) for v in r[3:18]] for r in rs])
        fo = np.array([np.longdouble(float(r[18])) for r in rs])
        fv, W = interpret(p, z, np.longdouble)
        kappa = (W / np.abs(fv)).astype(float)
        rel = np.abs((fv - fo) / fo).astype(float)
        good = kappa <= 1e4
        assert np.all(rel[good] <= 1e-12 + 16 * 2.0 ** -53 * kappa[good]), (gi, rel, kappa)
        n += int(good.sum())
    if n == 0:
        pytest.skip("no stored five-loop graph has a generated program")
