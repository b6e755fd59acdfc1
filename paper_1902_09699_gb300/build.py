"""Build libsip.so in-tree with nvcc for sm_103a (no CMake, no torch).

Each .cu translation unit is compiled to an object in parallel, then linked
into ``paper_1902_09699_gb300/libsip.so``.  ``build(guarded=True)`` also
compiles the kernels with the device index guards on (-DSIP_GUARDS) and
links them with the same host objects into ``libsip_guarded.so``, the debug
build that the binding loads when SIP_GUARDS=1.  Usage: ``python -m
paper_1902_09699_gb300.build [--guarded]`` or ``build()``.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libsip.so")
OUT_GUARDED = os.path.join(HERE, "libsip_guarded.so")
GUARDED = ["kernels.cu", "kernels_ml.cu"]  # the translation units with device index guards
BUILD = os.path.join(ROOT, "_build")
SOURCES = ["kernels.cu", "kernels_ml.cu", "api.cu", "handle.cu", "noalloc.cu", "server.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def build(verbose=False, guarded=False):
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include"),
                    "-I" + CSRC]
    procs = []
    objs = []
    gobjs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [cc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        if guarded and src in GUARDED:
            gobj = os.path.join(BUILD, src.replace(".cu", "_guarded.o"))
            gobjs.append(gobj)
            cmd = [cc] + flags + ["-DSIP_GUARDS", "-c", os.path.join(CSRC, src), "-o", gobj]
            procs.append((src + " (guarded)", subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        else:
            gobjs.append(obj)
    errs = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errs.append("%s:\n%s" % (src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    for out, ob in ((OUT, objs), (OUT_GUARDED, gobjs)) if guarded else ((OUT, objs),):
        tmp = out + ".tmp"
        cmd = [cc] + ARCH + ["-shared", "-o", tmp] + ob + ["-lcudart"]
        r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
        os.replace(tmp, out)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, guarded="--guarded" in sys.argv))
