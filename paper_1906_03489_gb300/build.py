"""Builds the spx shared library (sm_103a) in-tree: paper_1906_03489_gb300/lib/libspx.so.

Every translation unit is compiled by nvcc in parallel; the operator kernel
is compiled once per (precision, dimension, operator) from ``ops_inst.cu``.
Usage: ``python -m paper_1906_03489_gb300.build [--jobs N]``.
"""
import argparse
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libspx.so")
PROBE_LIB = os.path.join(LIBDIR, "libspx_probe.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]

OPS = range(8)


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def units():
    u = [("api", "api.cu", []), ("geom", "geom.cu", []), ("cg", "cg.cu", []),
         ("basis_host", "basis_host.cpp", [])]
    for tn in ("f64", "f32"):
        for dim in (2, 3):
            for op in OPS:
                u.append((f"ops_{tn}_{dim}_{op}", "ops_inst.cu",
                          [f"-DSPX_TN={tn}", f"-DSPX_DIM={dim}", f"-DSPX_OP={op}"]))
        for bk in (1, 2):   # 3D Helmholtz of the other basis kinds
            u.append((f"ops_{tn}_helm3_bk{bk}", "ops_inst.cu", [f"-DSPX_TN={tn}", f"-DSPX_BK={bk}"]))
        for cs in (1, 2, 3):   # triangles, prisms, tetrahedra
            u.append((f"collapsed_{tn}_{cs}", "collapsed.cu", [f"-DSPX_CT={tn}", f"-DSPX_CS={cs}"]))
    u.append(("collapsed_geom", "collapsed.cu", ["-DSPX_CGEOM"]))
    return u


# arithmetic-throughput probe of the benchmark: its own shared object
PROBE_UNITS = [("peak_probe", "peak_probe.cu", [])]


def source_digest():
    h = hashlib.sha256()
    for d in (CSRC, os.path.join(ROOT, "include")):
        for name in sorted(os.listdir(d)):
            with open(os.path.join(d, name), "rb") as f:
                h.update(name.encode() + f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    return h.hexdigest()


def compile_unit(nv, name, src, defs, verbose):
    obj = os.path.join(BUILD, name + ".o")
    cmd = [nv] + ARCH + NVCC_FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
    return obj, r.stderr


def build(jobs=None, force=False, verbose=False):
    """Compiles the library if its sources changed; returns the .so path."""
    digest = source_digest()
    stamp = os.path.join(LIBDIR, "libspx.sha256")
    if (not force and os.path.exists(LIB) and os.path.exists(PROBE_LIB) and os.path.exists(stamp)
            and open(stamp).read() == digest):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nv = nvcc()
    jobs = jobs or max(1, os.cpu_count() or 1)
    objs, logs = [], []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(compile_unit, nv, n, s, d, verbose) for n, s, d in units()]
        pfuts = [ex.submit(compile_unit, nv, n, s, d, verbose) for n, s, d in PROBE_UNITS]
        for f in futs:
            o, log = f.result()
            objs.append(o)
            logs.append(log)
        pobjs = []
        for f in pfuts:
            o, log = f.result()
            pobjs.append(o)
            logs.append(log)
    for out, obj_list in ((LIB, objs), (PROBE_LIB, pobjs)):
        tmp = out + ".tmp"
        cmd = [nv] + ARCH + ["-shared", "-o", tmp] + obj_list
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr)
        os.replace(tmp, out)
    with open(stamp, "w") as f:
        f.write(digest)
    if verbose:
        sys.stderr.write("".join(logs))
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=None)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--verbose", action="store_true", help="print ptxas register / spill reports")
    a = ap.parse_args()
    print(build(a.jobs, a.force, a.verbose))
