"""Build the native library in-tree: run the integrand generator, then nvcc.

    python -m paper_1905_08007_b300.build [--orders 1 2 3] [--programs 2 3 4] [--jobs 8]

Steps:
1. compile ``csrc/qed_gen.cpp`` with g++ and run it for the requested loop
   orders; it writes ``csrc/_gen/g_<id>.cuh`` (one device function per vertex
   graph, the forest-subtracted integrand) and ``csrc/_gen/qed_registry.h``;
2. compile one translation unit per graph (the kernels instantiated for that
   integrand) plus ``csrc/qedmc.cu`` (host side, C ABI, the interpreter
   kernels) for sm_103a, in parallel, and link them into ``libqedmc.so`` next
   to this file;
3. run the generator's bytecode back end for the program orders: it writes
   ``csrc/_gen/vm_n<n>.bin`` (one program per mirror-reduced graph; at five
   loops the 64 graphs of ``five_loop_subset.txt``, built only when asked
   for with ``--programs 2 3 4 5``, one generator process per graph and
   resumable), stored zlib-compressed as ``vm_n<n>.bin.z``; the library's
   interpreter kernels evaluate them (four loops and up have no compiled
   integrands; the lower orders are there to compare the two paths).
"""
from __future__ import annotations

import argparse
import re
import zlib
from concurrent.futures import ThreadPoolExecutor
import hashlib
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
GEN = CSRC / "_gen"
ROOT = PKG.parent
INCLUDE = ROOT / "include"
BUILD = ROOT / "_build"
LIB = PKG / "libqedmc.so"
DEFAULT_ORDERS = (1, 2, 3)
# five loops (the 64-graph workload of five_loop_subset.txt, hours and close
# to 60 GB of host memory to generate) only on request: --programs 2 3 4 5
DEFAULT_PROGRAM_ORDERS = (2, 3, 4)
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _run(cmd, **kw):
    print("+", " ".join(str(c) for c in cmd), flush=True)
    subprocess.run([str(c) for c in cmd], check=True, **kw)


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and Path(c).exists():
            return c
    raise RuntimeError("nvcc not found")


def _digest(paths, extra=""):
    h = hashlib.sha256(extra.encode())
    for p in paths:
        h.update(Path(p).read_bytes())
    return h.hexdigest()


GEN_SRC = [CSRC / "qed_gen.cpp", CSRC / "qed_graph.hpp", CSRC / "qed_vm_gen.hpp"]


def _generator():
    gen_bin = BUILD / "qed_gen"
    key = _digest(GEN_SRC)
    stamp = BUILD / "qed_gen.stamp"
    if not (gen_bin.exists() and stamp.exists() and stamp.read_text() == key):
        _run(["g++", "-O3", "-std=c++17", "-pthread", "-o", gen_bin, CSRC / "qed_gen.cpp"])
        stamp.write_text(key)
    return gen_bin


def _program_key(n):
    deps = GEN_SRC + ([PKG / "five_loop_subset.txt"] if n == 5 else [])
    return _digest(deps, extra=f"programs order {n}")


def build_programs(orders=DEFAULT_PROGRAM_ORDERS, force=False):
    """Bytecode programs vm_n<n>.bin.z for the interpreter kernels, one file
    and one stamp per loop order: an order is generated again only when its
    file is missing or the generator (or, at five loops, the graph list)
    changed, and the files of other orders are left alone."""
    orders = tuple(int(o) for o in orders)
    BUILD.mkdir(exist_ok=True)
    GEN.mkdir(exist_ok=True)
    todo = []
    keys = {n: _program_key(n) for n in orders}     # taken before generating
    for n in orders:
        out, stamp = GEN / f"vm_n{n}.bin.z", BUILD / f"programs_n{n}.stamp"
        if force or not (out.exists() and stamp.exists() and stamp.read_text() == keys[n]):
            todo.append(n)
    if 5 in todo:
        todo.remove(5)
        build_five_loop_programs(keys[5])
    if todo:
        for n in todo:
            for old in (GEN / f"vm_n{n}.bin", GEN / f"vm_n{n}.bin.z", BUILD / f"programs_n{n}.stamp"):
                if old.exists():
                    old.unlink()
        _run([_generator(), GEN] + [f"v{n}" for n in todo])
        for n in todo:
            compress_programs(GEN / f"vm_n{n}.bin")
            (BUILD / f"programs_n{n}.stamp").write_text(keys[n])
    return [GEN / f"vm_n{n}.bin.z" for n in orders]


def _program_records(path):
    """The program records of a generator file (after its 16-byte header)."""
    import struct
    data = Path(path).read_bytes()
    if data[:8] != b"QEDVM004":
        raise RuntimeError(f"{path}: not a program file")
    (n,) = struct.unpack_from("<I", data, 8)
    p, out = 16, []
    for _ in range(n):
        _, _, nins, nkon = struct.unpack_from("<4i", data, p + 64)
        size = 64 + 16 + 8 + 8 * nins + 8 * nkon
        out.append(data[p:p + size])
        p += size
    if p != len(data):
        raise RuntimeError(f"{path}: trailing bytes")
    return out


def build_five_loop_programs(key, jobs=None):
    """The 64-graph five-loop workload, one generator process per graph: a
    graph's forest expansion is released when its process ends (one process
    for all 64 graphs held every graph's working set and needed about 60 GB),
    and finished graphs are kept under _build/v5/ so that a rerun resumes.
    The programs are merged into vm_n5.bin.z in the order of
    five_loop_subset.txt; the stamp is written only when every graph is
    there (a partial file is still written and used)."""
    import struct
    subset = [int(x) for x in (PKG / "five_loop_subset.txt").read_text().split()]
    root = BUILD / "v5"
    root.mkdir(parents=True, exist_ok=True)
    gen = _generator()
    jobs = jobs or int(os.environ.get("QED_GEN_JOBS", "0")) or max(1, (os.cpu_count() or 2) // 2)

    def one(gi):
        d = root / f"g{gi}"
        done = d / "done.stamp"
        if done.exists() and done.read_text() == key and (d / "vm_n5.bin").exists():
            return gi, True
        d.mkdir(exist_ok=True)
        (d / "list.txt").write_text(f"{gi}\n")
        env = dict(os.environ, QED_GEN_JOBS="1")
        r = subprocess.run([str(gen), str(d), f"v5@{d / 'list.txt'}"], env=env, capture_output=True, text=True)
        ok = r.returncode == 0 and (d / "vm_n5.bin").exists() and len(_program_records(d / "vm_n5.bin")) == 1
        if ok:
            done.write_text(key)
        else:
            print(f"qed_gen: five-loop graph {gi} failed:\n{r.stderr[-2000:]}", flush=True)
        return gi, ok

    print(f"+ five-loop programs: {len(subset)} graphs, {jobs} generator processes", flush=True)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        status = dict(ex.map(one, subset))
    blobs = [_program_records(root / f"g{gi}" / "vm_n5.bin")[0] for gi in subset if status[gi]]
    raw = GEN / "vm_n5.bin"
    raw.write_bytes(b"QEDVM004" + struct.pack("<2I", len(blobs), 0) + b"".join(blobs))
    compress_programs(raw)
    stamp = BUILD / "programs_n5.stamp"
    if len(blobs) == len(subset):
        stamp.write_text(key)
    elif stamp.exists():
        stamp.unlink()
    print(f"+ five-loop programs: {len(blobs)} of {len(subset)} graphs", flush=True)


def compress_programs(raw):
    """vm_n<n>.bin -> vm_n<n>.bin.z (zlib; programs shrink about 6x)."""
    raw = Path(raw)
    z = raw.with_name(raw.name + ".z")
    z.write_bytes(zlib.compress(raw.read_bytes(), 6))
    raw.unlink()
    return z


def build(orders=DEFAULT_ORDERS, force=False, verbose_ptxas=False, jobs=None,
          program_orders=DEFAULT_PROGRAM_ORDERS):
    lib = build_library(orders, force, verbose_ptxas, jobs)
    build_programs(program_orders, force)
    return lib


def build_library(orders=DEFAULT_ORDERS, force=False, verbose_ptxas=False, jobs=None):
    orders = tuple(int(o) for o in orders)
    BUILD.mkdir(exist_ok=True)
    GEN.mkdir(exist_ok=True)
    lib_src = [CSRC / "qedmc.cu", CSRC / "qed_kernels.cuh", CSRC / "qed_batch.cuh", CSRC / "qed_dd.cuh",
               CSRC / "qed_vm.cuh", CSRC / "qed_graph.hpp", INCLUDE / "qedmc.h"]
    stamp = BUILD / "libqedmc.stamp"
    key = _digest(GEN_SRC + lib_src, extra=repr(orders) + ARCH + repr(verbose_ptxas))
    if not force and LIB.exists() and stamp.exists() and stamp.read_text() == key:
        return LIB
    gen_bin = _generator()
    for pat in ("g_*.cuh", "k_*.cu", "qed_registry.h"):
        for old in GEN.glob(pat):
            old.unlink()
    _run([gen_bin, GEN] + list(orders))
    reg = (GEN / "qed_registry.h").read_text()
    ids = re.findall(r"X\((\d+), (\d+)\)", reg.split("QED_GENERATED_LIST(X)")[1].splitlines()[0])
    objdir = BUILD / "obj"
    objdir.mkdir(exist_ok=True)
    big = [(gid, ln) for gid, ln in ids if int(ln) >= 9]      # three loops and up
    rdc = bool(big)
    base = [_nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
            "--expt-relaxed-constexpr", "-I", INCLUDE, "-I", CSRC, "-I", GEN]
    if rdc:
        base.append("-rdc=true")
    if verbose_ptxas:
        base.append("-Xptxas=-v")
    units = []
    bigset = {gid for gid, _ in big}
    kern_h = [CSRC / "qed_kernels.cuh", CSRC / "qed_dd.cuh"]
    for gid, lines in ids:
        tu = GEN / f"k_{gid}.cu"
        text = f'#include "qed_kernels.cuh"\n#include "g_{gid}.cuh"\nQED_DEFINE_KSET({gid}, {lines})\n'
        if gid in bigset:
            # the integrand once per precision, for the batched kernels to link against
            text += (f"__device__ double qed_ext_f64_{gid}(const double* z, double& a) "
                     f"{{ return qed_gen_f<{gid}>::template eval<double>(z, a); }}\n"
                     f"__device__ dd qed_ext_dd_{gid}(const dd* z, double& a) "
                     f"{{ return qed_gen_f<{gid}>::template eval<dd>(z, a); }}\n")
        tu.write_text(text)
        units.append((tu, objdir / f"k_{gid}.o", kern_h + [GEN / f"g_{gid}.cuh"]))
    # the persistent batched kernels: one switch over every generated graph;
    # graphs of three loops and up are linked in (relocatable device code)
    # rather than compiled again here
    btu = GEN / "k_batch.cu"
    inc = ""
    for gid, _ in ids:
        if gid not in bigset:
            inc += f'#include "g_{gid}.cuh"\n'
        else:
            inc += (f"extern __device__ double qed_ext_f64_{gid}(const double*, double&);\n"
                    f"extern __device__ dd qed_ext_dd_{gid}(const dd*, double&);\n"
                    f"template <> struct qed_gen_f<{gid}> {{\n"
                    f"  template <class R> __device__ static R eval(const R* z, double& a);\n}};\n"
                    f"template <> template <> __device__ double qed_gen_f<{gid}>::eval<double>(const double* z, double& a) "
                    f"{{ return qed_ext_f64_{gid}(z, a); }}\n"
                    f"template <> template <> __device__ dd qed_gen_f<{gid}>::eval<dd>(const dd* z, double& a) "
                    f"{{ return qed_ext_dd_{gid}(z, a); }}\n")
    c64 = " ".join(f"case {gid}: batch_item_fp64<{gid}, {ln}>(B, it, I, smem); break;" for gid, ln in ids)
    cdd = " ".join(f"case {gid}: batch_item_dd<{gid}, {ln}>(B, it, I, smem); break;" for gid, ln in ids)
    btu.write_text(
        f'#define QED_BATCH_TU 1\n#include "qed_batch.cuh"\n{inc}'
        f'__device__ void batch_dispatch_fp64(const BatchParams &B, unsigned int it, const BatchItem &I, double *smem) {{\n'
        f'  switch (B.diags[I.diag].fid) {{ {c64} default: break; }}\n}}\n'
        f'__device__ void batch_dispatch_dd(const BatchParams &B, unsigned int it, const BatchItem &I, double *smem) {{\n'
        f'  switch (B.diags[I.diag].fid) {{ {cdd} default: break; }}\n}}\n')
    units.append((btu, objdir / "k_batch.o",
                  kern_h + [CSRC / "qed_batch.cuh"] + [GEN / f"g_{gid}.cuh" for gid, _ in ids if gid not in bigset]))
    units.append((CSRC / "qedmc.cu", objdir / "qedmc.o",
                  sorted(CSRC.glob("*.cuh")) + [CSRC / "qed_graph.hpp", INCLUDE / "qedmc.h", GEN / "qed_registry.h"]))

    def compile_one(u):
        # an object is reused when its source, the headers it includes and
        # the flags are unchanged
        src, obj, deps = u
        cmd = base + ["-c", "-o", obj, src]
        okey = _digest([src] + list(deps), extra=" ".join(str(c) for c in cmd))
        ostamp = obj.with_suffix(".stamp")
        if obj.exists() and ostamp.exists() and ostamp.read_text() == okey:
            return src, ""
        r = subprocess.run([str(c) for c in cmd], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        ostamp.write_text(okey)
        return src, r.stderr

    jobs = jobs or max(1, os.cpu_count() or 1)
    print(f"+ nvcc {len(units)} translation units, {jobs} jobs", flush=True)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        for src, err in ex.map(compile_one, units):
            if verbose_ptxas and err:
                print(f"== {src.name}\n{err}")
    keep = {o for _, o, _ in units}
    for old in objdir.glob("*.o"):
        if old not in keep:
            old.unlink()
    _run([_nvcc(), ARCH, "-shared"] + (["-rdc=true"] if rdc else []) + ["-o", LIB] +
         [o for _, o, _ in units] + ["-lcudart"])
    stamp.write_text(key)
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--orders", nargs="*", type=int, default=list(DEFAULT_ORDERS))
    ap.add_argument("--programs", nargs="*", type=int, default=list(DEFAULT_PROGRAM_ORDERS))
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--ptxas-v", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    a = ap.parse_args(argv)
    print(build(a.orders, force=a.force, verbose_ptxas=a.ptxas_v, jobs=a.jobs, program_orders=a.programs))


if __name__ == "__main__":
    sys.exit(main())
