"""Program files of the generator's bytecode back end, one stamp per loop
order (paper_1905_08007_b300/build.py): an order is generated only when its
file or stamp is missing or stale, and building one order leaves the files
of the others alone.  Runs the generator for two loops only (seconds), into
a temporary directory."""
import pytest

from paper_1905_08007_b300 import build as b


@pytest.fixture
def tmp_build(tmp_path, monkeypatch):
    gen = b.BUILD / "qed_gen"
    if not gen.exists():
        pytest.skip("generator not built (run the package build first)")
    monkeypatch.setattr(b, "GEN", tmp_path / "gen")
    monkeypatch.setattr(b, "BUILD", tmp_path / "build")
    monkeypatch.setattr(b, "_generator", lambda: gen)
    calls = []
    real_run = b._run

    def run(cmd, **kw):
        calls.append([str(c) for c in cmd])
        return real_run(cmd, **kw)
    monkeypatch.setattr(b, "_run", run)
    return tmp_path, calls


def test_each_order_has_its_own_stamp(tmp_build):
    tmp, calls = tmp_build
    out = b.build_programs((2,))
    assert out == [tmp / "gen" / "vm_n2.bin.z"] and out[0].exists()
    assert not (tmp / "gen" / "vm_n2.bin").exists()
    assert (tmp / "build" / "programs_n2.stamp").read_text() == b._program_key(2)
    assert len(calls) == 1 and calls[0][-1] == "v2"
    data = out[0].read_bytes()
    # unchanged generator and file: nothing runs again
    b.build_programs((2,))
    assert len(calls) == 1
    # a stale stamp regenerates that order only
    (tmp / "build" / "programs_n2.stamp").write_text("stale")
    b.build_programs((2,))
    assert len(calls) == 2 and calls[1][-1] == "v2"
    assert out[0].read_bytes() == data          # the generator is deterministic


def test_five_loop_programs_are_not_in_the_default_build():
    assert 5 not in b.DEFAULT_PROGRAM_ORDERS and 4 in b.DEFAULT_PROGRAM_ORDERS
    assert b._program_key(5) != b._program_key(4)
