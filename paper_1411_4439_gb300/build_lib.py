"""Build libhisq.so in-tree for sm_103a (GB300) with nvcc.

Every translation unit compiles in parallel; the Dslash kernel families are
one source (csrc/dslash_inst.cu) compiled once per (storage precision, fat
link compression, Naik link compression). Objects go to _build/ beside this
file, the library to lib/libhisq.so. Nothing is rebuilt when the library is
newer than every source.

    python -m paper_1411_4439_gb300.build_lib [--force] [--jobs N]
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB_DIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIB_DIR, "libhisq.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           f"-I{INCLUDE}", f"-I{CSRC}"]

# (object name, defines) of the Dslash families
FAMILIES = [
    ("dslash_f64_18_18", dict(HISQ_STORE="double", HISQ_LSTORE="double", HISQ_RU=18, HISQ_RN=18, HISQ_MAX_RPT=4, HISQ_WITH_XY=1)),
    ("dslash_f32_18_18", dict(HISQ_STORE="float", HISQ_LSTORE="float", HISQ_RU=18, HISQ_RN=18, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f32_18_14", dict(HISQ_STORE="float", HISQ_LSTORE="float", HISQ_RU=18, HISQ_RN=14, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f32_12_14", dict(HISQ_STORE="float", HISQ_LSTORE="float", HISQ_RU=12, HISQ_RN=14, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f32_14_14", dict(HISQ_STORE="float", HISQ_LSTORE="float", HISQ_RU=14, HISQ_RN=14, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f16_18_18", dict(HISQ_STORE="__half", HISQ_LSTORE="hisq::Fx16", HISQ_RU=18, HISQ_RN=18, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f16_18_14", dict(HISQ_STORE="__half", HISQ_LSTORE="hisq::Fx16", HISQ_RU=18, HISQ_RN=14, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f16_12_14", dict(HISQ_STORE="__half", HISQ_LSTORE="hisq::Fx16", HISQ_RU=12, HISQ_RN=14, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
    ("dslash_f16_14_14", dict(HISQ_STORE="__half", HISQ_LSTORE="hisq::Fx16", HISQ_RU=14, HISQ_RN=14, HISQ_MAX_RPT=8, HISQ_WITH_XY=0)),
]
PLAIN = ["hisq_api", "dslash_dispatch", "gauge", "blas", "blas_bundle", "force", "noalloc"]
# bundle-layout Dslash families (FP32 / FP16 storage); the U r18 / N r14 ones
# carry every mapping the autotuner chooses from
BUNDLE_FAMILIES = [(name, defs, 1 if (defs["HISQ_RU"], defs["HISQ_RN"]) == (18, 14) else 0)
                   for name, defs in FAMILIES if defs["HISQ_STORE"] != "double"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhisq")


def _sources():
    out = []
    for root, _, files in os.walk(CSRC):
        out += [os.path.join(root, f) for f in files if f.endswith((".cu", ".cuh", ".h"))]
    out += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return out


def _up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources() + [os.path.abspath(__file__)])


def _compile(args):
    cmd, obj = args
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {obj}:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    return obj


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    """Compile every CUDA unit and link lib/libhisq.so; returns the library path."""
    if not force and _up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIB_DIR, exist_ok=True)
    tasks = []
    for name in PLAIN:
        obj = os.path.join(BUILD, name + ".o")
        tasks.append(([nvcc, *ARCH, *NVFLAGS, "-c", os.path.join(CSRC, name + ".cu"), "-o", obj], obj))
    for name, defs in FAMILIES:
        for layout, suffix in ((0, "aos"), (1, "soa")):
            obj = os.path.join(BUILD, f"{name}_{suffix}.o")
            dflags = [f"-D{k}={v}" for k, v in defs.items()]
            dflags += [f"-DHISQ_FAMILY={name}_{suffix}", f"-DHISQ_LAYOUT={layout}"]
            tasks.append(([nvcc, *ARCH, *NVFLAGS, *dflags, "-c", os.path.join(CSRC, "dslash_inst.cu"),
                           "-o", obj], obj))
    for name, defs, full in BUNDLE_FAMILIES:
        obj = os.path.join(BUILD, f"{name}_bundle.o")
        dflags = [f"-D{k}={v}" for k, v in defs.items() if k in ("HISQ_STORE", "HISQ_LSTORE", "HISQ_RU", "HISQ_RN")]
        dflags += [f"-DHISQ_FAMILY={name}_bundle", f"-DHISQ_BUNDLE_FULL={full}"]
        tasks.append(([nvcc, *ARCH, *NVFLAGS, *dflags, "-c", os.path.join(CSRC, "dslash_bundle_inst.cu"),
                       "-o", obj], obj))
    # longest compiles first
    tasks.sort(key=lambda t: 0 if "_bundle.o" in t[1] else 1)
    jobs = jobs or min(len(tasks), max(1, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(_compile, tasks))
    tmp = LIB + ".tmp"
    link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fPIC"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{' '.join(link)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        print(f"built {LIB}")
    return LIB


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--force", action="store_true")
    ap.add_argument("--jobs", type=int, default=None)
    a = ap.parse_args(argv)
    print(build(force=a.force, jobs=a.jobs, verbose=True))


if __name__ == "__main__":
    sys.exit(main())
