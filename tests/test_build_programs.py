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


FAKE_GEN = r'''#!/usr/bin/env python3
# stand-in for qed_gen's five-loop back end: "<dir> v5@<list>" writes one
# program record per listed graph (name g<index>, a single END word); the
# graph whose index is in FAIL exits 1 without writing
import os, struct, sys
d, arg = sys.argv[1], sys.argv[2]
idx = [int(x) for x in open(arg.split("@", 1)[1]).read().split()]
fail = {int(x) for x in os.environ.get("FAKE_FAIL", "").split()}
if set(idx) & fail:
    sys.exit(1)
with open(os.path.join(d, "vm_n5.bin"), "wb") as f:
    f.write(b"QEDVM004" + struct.pack("<2I", len(idx), 0))
    for i in idx:
        f.write(f"g{i}".encode().ljust(64, b"\0") + struct.pack("<4i", 15, 15, 1, 0) + struct.pack("<d", 0.0))
        f.write(struct.pack("<Q", 4 << 34))
'''


def test_five_loop_programs_one_process_per_graph_resume_and_partial(tmp_path, monkeypatch):
    """--programs 5 runs one generator process per graph, merges the
    finished ones in the workload's order, writes the stamp only when all
    are there, and a rerun generates only the missing graphs."""
    import zlib
    gen = tmp_path / "fake_gen"
    gen.write_text(FAKE_GEN)
    gen.chmod(0o755)
    pkg = tmp_path / "pkg"
    pkg.mkdir()
    (pkg / "five_loop_subset.txt").write_text("91 7 158\n")
    monkeypatch.setattr(b, "PKG", pkg)
    monkeypatch.setattr(b, "GEN", tmp_path / "gen")
    monkeypatch.setattr(b, "BUILD", tmp_path / "build")
    monkeypatch.setattr(b, "_generator", lambda: gen)
    (tmp_path / "gen").mkdir()
    calls = []
    real = b.subprocess.run

    def run(cmd, **kw):
        calls.append(cmd)
        return real(cmd, **kw)
    monkeypatch.setattr(b.subprocess, "run", run)
    key = "k1"

    def names():
        data = zlib.decompress((tmp_path / "gen" / "vm_n5.bin.z").read_bytes())
        return [r[:64].split(b"\0")[0].decode() for r in [data[16 + i * 96:16 + (i + 1) * 96]
                                                          for i in range(struct_count(data))]]
    monkeypatch.setenv("FAKE_FAIL", "7")
    b.build_five_loop_programs(key, jobs=2)
    assert names() == ["g91", "g158"] and not (tmp_path / "build" / "programs_n5.stamp").exists()
    assert len(calls) == 3
    monkeypatch.setenv("FAKE_FAIL", "")
    b.build_five_loop_programs(key, jobs=2)
    assert len(calls) == 4                                  # only graph 7 again
    assert names() == ["g91", "g7", "g158"]
    assert (tmp_path / "build" / "programs_n5.stamp").read_text() == key


def struct_count(data):
    import struct
    return struct.unpack_from("<I", data, 8)[0]
