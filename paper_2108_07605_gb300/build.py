"""Build the CUDA library in-tree for sm_103a.

    python -m paper_2108_07605_gb300.build [--force]

Compiles every translation unit of csrc/ with nvcc in parallel and links
_lib/libpaper2108lbm.so.  Outputs are rebuilt when a source or header is
newer than the library.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIBNAME = "libpaper2108lbm.so"
LIBPATH = os.path.join(LIBDIR, LIBNAME)
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# (source, object, defines): the kernel templates are instantiated once per
# (lattice, species count, precision) in their own translation unit, so the
# longest compile is one instantiation, not all of them
UNITS = [("lbm_capi.cu", "lbm_capi.o", []),
         ("lbm_noalloc.cu", "lbm_noalloc.o", []),
         ("lbm_probe.cu", "lbm_probe.o", []),
         ("lbm_dispatch.cu", "lbm_dispatch.o", [])]
for _d, _m in ((3, 9), (3, 2), (2, 9), (2, 2)):
    for _prec, _tag in ((0, "f64"), (1, "f32"), (2, "f16"), (3, "c64")):
        UNITS.append(("lbm_inst.cu", f"lbm_inst_{_d}_{_m}_{_tag}.o",
                      [f"-DLBM_D={_d}", f"-DLBM_M={_m}", f"-DLBM_PREC={_prec}",
                       f"-DLBM_CHEM64={1 if _prec == 3 else 0}",
                       f"-DLBM_KSET=kernel_set_{_d}_{_m}_{_tag}"]))


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "lbm.h"))
    return files


def _stale():
    if not os.path.exists(LIBPATH):
        return True
    t = os.path.getmtime(LIBPATH)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force=False, verbose=False):
    """Compile and link; returns the library path."""
    if not force and not _stale():
        return LIBPATH
    os.makedirs(LIBDIR, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-I", os.path.join(ROOT, "include"), "--expt-relaxed-constexpr"]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(unit):
        src, objname, defs = unit
        obj = os.path.join(LIBDIR, objname)
        cmd = [cc] + common + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {objname}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    # the longest units first
    order = sorted(UNITS, key=lambda u: ("_3_9_" not in u[1], "lbm_inst" not in u[1]))
    workers = max(1, min(len(UNITS), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        results = list(ex.map(compile_one, order))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results]
    tmp = LIBPATH + ".tmp"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIBPATH)
    return LIBPATH


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIBPATH)
