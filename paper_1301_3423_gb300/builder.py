"""Build librlb.so in-tree for sm_103a.

Steps: generate the compile-time quadrature header from lattice/*.txt, compile the C-ABI unit and
one kernel-instantiation unit per (order, storage) in parallel with nvcc, link a shared library
into paper_1301_3423_gb300/_build/.  The build is skipped when the sources, the lattice files and
the flags are unchanged (content hash)."""
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "librlb.so")
INCLUDE = os.path.join(ROOT, "include")
LATTICE = os.path.join(ROOT, "lattice")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v"]
INSTANCES = [(o, s) for o in (3, 2) for s in (0, 1, 2)]
# step-kernel variants compiled per (order, storage): one for double storage, four for float ones
VARIANT_UNITS = [(o, s, v) for o, s in INSTANCES for v in ((0,) if s == 0 else (0, 1, 2, 3))]
# pipelined step kernel per (order, storage), tile width and tile kind (row tiles: widths 128 and 96)
PIPE_UNITS = [(o, s, tx, rows) for o, s in INSTANCES for tx, rows in ((64, 0), (128, 0), (128, 1), (96, 1))]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _sources():
    files = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh", ".h", ".py")))
    files += [os.path.join(INCLUDE, "rlb.h"), os.path.join(LATTICE, "d3q128.txt"), os.path.join(LATTICE, "d3q66.txt")]
    return files


def _digest():
    h = hashlib.sha256(" ".join(NVCC_FLAGS).encode())
    for f in _sources():
        h.update(f.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def build(force=False, verbose=False):
    """Compile librlb.so if needed; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "librlb.sha256")
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp) and open(stamp).read().strip() == digest:
        return LIB
    sys.path.insert(0, CSRC)
    try:
        import gen_quadrature
    finally:
        sys.path.pop(0)
    gen_quadrature.main(LATTICE, os.path.join(BUILD, "rlb_quadrature.h"))
    nvcc = _nvcc()
    inc = ["-I", INCLUDE, "-I", BUILD, "-I", CSRC]
    jobs = [(os.path.join(BUILD, "rlb_api.o"), [nvcc] + NVCC_FLAGS + inc + ["-c", os.path.join(CSRC, "rlb_api.cu")])]
    jobs.append((os.path.join(BUILD, "rlb_batch.o"), [nvcc] + NVCC_FLAGS + inc + [
        "-c", os.path.join(CSRC, "rlb_batch.cu"), "-o", os.path.join(BUILD, "rlb_batch.o")]))
    jobs.append((os.path.join(BUILD, "rlb_noalloc.o"), [nvcc] + NVCC_FLAGS + inc + [
        "-c", os.path.join(CSRC, "rlb_noalloc.cu"), "-o", os.path.join(BUILD, "rlb_noalloc.o")]))
    for o, s in INSTANCES:
        obj = os.path.join(BUILD, "rlb_inst_o%d_s%d.o" % (o, s))
        jobs.append((obj, [nvcc] + NVCC_FLAGS + inc + ["-DRLB_INST_ORDER=%d" % o, "-DRLB_INST_STORAGE=%d" % s,
                                                          "-c", os.path.join(CSRC, "rlb_inst.cu"), "-o", obj]))
    for o, s, v in VARIANT_UNITS:
        obj = os.path.join(BUILD, "rlb_inst_o%d_s%d_v%d.o" % (o, s, v))
        jobs.append((obj, [nvcc] + NVCC_FLAGS + inc + ["-DRLB_INST_ORDER=%d" % o, "-DRLB_INST_STORAGE=%d" % s,
                                                          "-DRLB_INST_VARIANT=%d" % v, "-c",
                                                          os.path.join(CSRC, "rlb_inst_variant.cu"), "-o", obj]))
    for o, s, tx, rows in PIPE_UNITS:
        obj = os.path.join(BUILD, "rlb_inst_o%d_s%d_%s%d.o" % (o, s, "r" if rows else "x", tx))
        jobs.append((obj, [nvcc] + NVCC_FLAGS + inc + ["-DRLB_INST_ORDER=%d" % o, "-DRLB_INST_STORAGE=%d" % s,
                                                          "-DRLB_INST_TX=%d" % tx, "-DRLB_INST_ROWS=%d" % rows, "-c",
                                                          os.path.join(CSRC, "rlb_inst_pipe.cu"), "-o", obj]))
    # longest units first so the parallel build ends sooner
    jobs = jobs[:1] + sorted(jobs[1:], key=lambda j: ("_v" not in j[0], "_s0" in j[0]))
    jobs[0][1].extend(["-o", jobs[0][0]])
    logs = []
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), max(os.cpu_count() or 4, 4))) as ex:
        for out in ex.map(lambda j: _run(j[1]), jobs):
            logs.append(out)
    tmp = LIB + ".%d.tmp" % os.getpid()
    _run([nvcc] + ARCH + ["-shared", "-o", tmp] + [j[0] for j in jobs] + ["-lcudart"])
    os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write("\n".join(logs))
    with open(stamp, "w") as fh:
        fh.write(digest)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
