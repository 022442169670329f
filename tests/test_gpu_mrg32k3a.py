"""MRG32k3a (Sec. 3, Calc 1) on the GPU through the C ABI.

* The oracle's recurrence against the MRG32k3a of the CURAND library, the
  generator the paper ran: a small CUDA program (compiled here with nvcc
  against CURAND's device header) sets CURAND's state to the oracle's state
  and returns its raw outputs, which must equal the oracle's z values
  exactly, from the all-12345 state and from a state after a jump of about
  2^130 steps.
* The library's points, log p and sector decisions with MRG32k3a draws
  against the oracle's sampler fed by the oracle's MRG32k3a, at counters
  near 0 and near 1e8 (jumps over many index bits), for the one-loop graph
  and two two-loop graphs, to 1e-12 (as for Philox).
* The batched path equals the per-graph path on the same counters with
  MRG32k3a, and the generators are independent checks of one integral:
  the one-loop value 1/2 and the two-loop set total within 3 sigma from
  each generator, and the two estimates combined by inverse variance as
  Sec. 3 combines Calc 1 and Calc 2.
"""
import math
import shutil
import subprocess
import textwrap

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1905_08007_b300 as q                     # noqa: E402
from oracle import mrg32k3a as om                      # noqa: E402
from oracle.graphs import deg_table, enumerate_graphs as o_enum   # noqa: E402
from oracle.pdf import f_table, sample_points          # noqa: E402
from oracle.estimator import combine_inverse_variance  # noqa: E402

TWO_LOOP = -0.34416638743829586

CURAND_PROBE = textwrap.dedent(r"""
    #include <cstdio>
    #include <cstdlib>
    #include <curand_kernel.h>
    __global__ void k(unsigned int a0, unsigned int a1, unsigned int a2, unsigned int b0,
                      unsigned int b1, unsigned int b2, int n, double *out) {
      curandStateMRG32k3a_t st;
      st.s1[0] = a0; st.s1[1] = a1; st.s1[2] = a2;
      st.s2[0] = b0; st.s2[1] = b1; st.s2[2] = b2;
      st.boxmuller_flag = 0; st.boxmuller_flag_double = 0;
      for (int i = 0; i < n; ++i) out[i] = curand_MRG32k3a(&st);
    }
    int main(int argc, char **argv) {
      unsigned int s[6];
      for (int i = 0; i < 6; ++i) s[i] = (unsigned int)strtoul(argv[1 + i], 0, 10);
      const int n = atoi(argv[7]);
      double *d, *h = (double *)malloc(n * sizeof(double));
      if (cudaMalloc(&d, n * sizeof(double)) != cudaSuccess) return 2;
      k<<<1, 1>>>(s[0], s[1], s[2], s[3], s[4], s[5], n, d);
      if (cudaMemcpy(h, d, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
      for (int i = 0; i < n; ++i) printf("%.1f\n", h[i]);
      cudaFree(d);
      return 0;
    }
""")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tmp_path_factory.mktemp("curand")
    src = d / "probe.cu"
    src.write_text(CURAND_PROBE)
    exe = d / "probe"
    subprocess.run([nvcc, "-gencode=arch=compute_103a,code=sm_103a", "-O2", "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    return exe


def _oracle_z(s1, s2, n):
    out = []
    for _ in range(n):
        p1 = (om.A12 * s1[1] - om.A13 * s1[0]) % om.M1
        p2 = (om.A21 * s2[2] - om.A23 * s2[0]) % om.M2
        s1, s2, u = om.step(s1, s2)
        z = (p1 - p2) % om.M1
        out.append(z if z > 0 else om.M1)
        assert u == float(out[-1]) * om.NORM
    return out


@pytest.mark.parametrize("pos", [0, (3 << 127) + (5 << 96) + (123456789 << 5)])
def test_oracle_recurrence_equals_curand(probe, pos):
    s1, s2 = om.state_at(pos)
    n = 2000
    r = subprocess.run([str(probe)] + [str(v) for v in (*s1, *s2)] + [str(n)], check=True,
                       capture_output=True, text=True)
    got = [int(float(x)) for x in r.stdout.split()]
    assert got == _oracle_z(s1, s2, n)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return q.Context(0, threshold=1e-12, rng="mrg32k3a")


@pytest.mark.parametrize("n,gi", [(1, 0), (2, 1), (2, 4)])
@pytest.mark.parametrize("begin,count,seed", [(0, 517, 0), (10**8 - 211, 211, 7)])
def test_points_and_density_match_oracle(ctx, n, gi, begin, count, seed):
    g = q.enumerate_graphs(n)[gi]
    og = o_enum(n)[gi]
    d = ctx.load(g)
    z, f, lp, fl = d.dump_points(begin, count, seed=seed)
    z, lp = z.cpu().numpy(), lp.cpu().numpy()
    N = og.n_lines
    deg = deg_table(og)
    u = om.uniforms(np.arange(begin, begin + count, dtype=np.uint64), g.stream_id, seed, 2 * (N - 1))
    xo, lpo, _ = sample_points(u, deg, f_table(deg, N), N)
    assert np.array_equal(np.argsort(-z, axis=1, kind="stable"), np.argsort(-xo, axis=1, kind="stable"))
    np.testing.assert_allclose(z, xo, rtol=1e-12, atol=0)
    np.testing.assert_allclose(lp, lpo, rtol=1e-12, atol=1e-12)


def test_generators_draw_different_points(ctx):
    g = q.enumerate_graphs(2)[1]
    zm = ctx.load(g).dump_points(0, 64, seed=0)[0].cpu().numpy()
    cp = q.Context(0, threshold=1e-12)
    zp = cp.load(g).dump_points(0, 64, seed=0)[0].cpu().numpy()
    assert not np.allclose(zm, zp)


def test_batch_equals_per_graph_with_mrg():
    c = q.Context(0, rng="mrg32k3a")
    ds = [c.load(g) for g in q.enumerate_graphs(2)[:3]]
    res = c.integrate_batch(ds, 3 * (1 << 20), seed=3, policy="equal", rounds=2, chunk=1 << 18)
    for d, r in zip(ds, res):
        one = d.integrate(r.n, seed=3)
        assert one.n == r.n
        assert one.value == pytest.approx(r.value, rel=1e-9, abs=1e-13)


def test_calc1_and_calc2_agree_with_the_closed_forms():
    """One- and two-loop totals from each generator within 3 sigma of the
    closed forms; the two estimates combined by inverse variance (Sec. 3)."""
    vals = {}
    for rng in ("mrg32k3a", "philox"):
        c = q.Context(0, rng=rng)
        r1 = c.load(q.enumerate_graphs(1)[0]).integrate(4_000_000, seed=11)
        assert abs(r1.value - 0.5) < 3 * r1.sigma + 1e-12, (rng, r1.value, r1.sigma)
        ds = [c.load(g) for g in q.enumerate_graphs(2)]
        for d in ds:
            d.calibrate_deg(n_base=8, seed=5)
        res = c.integrate_batch(ds, 6 * 10**7, seed=11, policy="variance", rounds=4, chunk=1 << 18)
        tot = sum(r.value for r in res)
        sig = math.sqrt(sum(r.variance for r in res))
        assert abs(tot - TWO_LOOP) < 3 * sig, (rng, tot, sig)
        vals[rng] = (tot, sig)
    (a, sa), (b, sb) = vals["mrg32k3a"], vals["philox"]
    assert abs(a - b) < 3 * math.hypot(sa, sb)
    v, s = combine_inverse_variance([a, b], [sa, sb])
    assert abs(v - TWO_LOOP) < 3 * s
