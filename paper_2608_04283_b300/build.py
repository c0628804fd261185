"""Build the CUDA libraries in-tree with nvcc for sm_103a.

  libvklb.so            the simulation library (C ABI of include/vklb.h)
  libvklb_hostcheck.so  host-only evaluation of the closed-form splits, used by
                        CPU tests to compare them with the FP64 oracle

Usage: python -m paper_2608_04283_b300.build  (or build() from Python).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

LIB = os.path.join(HERE, "libvklb.so")
HOSTCHECK = os.path.join(HERE, "libvklb_hostcheck.so")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))] + [os.path.join(INCLUDE, "vklb.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed: " + " ".join(cmd))
    return res


# translation units of libvklb.so: the C ABI and one per system's kernels
UNITS = ["vklb.cu", "ops_advect.cu", "ops_swe.cu", "ops_euler.cu", "ops_mhd.cu", "ops_mhd_fp64.cu",
         "ops_mhd_fp32.cu", "ops_mhd_bf16.cu"]


def build(force=False, verbose=False):
    deps = _sources()
    if force or _stale(LIB, deps):
        objdir = os.path.join(HERE, "_build")
        os.makedirs(objdir, exist_ok=True)
        cmds = []
        for u in UNITS:
            cmd = [NVCC, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-c", "-I" + INCLUDE,
                   "-o", os.path.join(objdir, u + ".o"), os.path.join(CSRC, u)]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            cmds.append(cmd)
        with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
            list(ex.map(_run, cmds))
        _run([NVCC, *ARCH, "-shared", "-o", LIB] + [os.path.join(objdir, u + ".o") for u in UNITS])
    if force or _stale(HOSTCHECK, deps):
        cmd = [NVCC, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-I" + INCLUDE,
               "-o", HOSTCHECK, os.path.join(CSRC, "hostcheck.cu")]
        _run(cmd)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
