"""Build the LEAD C-ABI library (liblead.so) in-tree for sm_103a.

Translation units are compiled in parallel with nvcc (CUDA) and g++ (host construction), then
linked into ``paper_2605_17796_gb300/liblead.so``. Run ``python -m paper_2605_17796_gb300.build``.
``--checked`` builds ``liblead_checked.so`` instead (LEAD_CHECKED: kernels test their table-driven
indices and entry points report failures as LEAD_ECHECK), in its own build folder.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "liblead.so")
LIB_CHECKED = os.path.join(HERE, "liblead_checked.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CU_SOURCES = ["device.cu", "sample.cu", "decode.cu", "priors.cu", "prior_tc.cu", "local.cu", "osd.cu",
              "iterated.cu"]
CPP_SOURCES = ["code.cpp", "jit.cpp", "server.cpp"]
# the run-time specialised min-sum kernel: these files are embedded (in this order) as text
JIT_SOURCES = ["bp_jit_args.h", "lead_llr.cuh", "lead_math.cuh", "bp_jit_kernel.cuh"]
CUDA_HOME = "/usr/local/cuda"


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the LEAD library needs the CUDA toolkit to build")


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def _write_jit_source(build_dir: str = BUILD):
    """Embed the specialised kernel's source as a C++ raw string (lead_jit_source.inc)."""
    parts = []
    for name in JIT_SOURCES:
        text = open(os.path.join(CSRC, name)).read()
        # the files come concatenated in dependency order: drop the guards and the local includes
        text = "\n".join(line for line in text.splitlines()
                         if line.strip() != "#pragma once" and not line.startswith('#include "'))
        parts.append(f"// ---- {name}\n{text}\n")
    body = "".join(parts)
    if ")LEADJIT" in body:
        raise RuntimeError("kernel source contains the raw-string delimiter")
    out = os.path.join(build_dir, "lead_jit_source.inc")
    new = 'static const char kLeadJitSource[] = R"LEADJIT(\n' + body + ')LEADJIT";\n'
    if not os.path.exists(out) or open(out).read() != new:
        with open(out, "w") as f:
            f.write(new)


def build(verbose: bool = False, ptxas_info: bool = False, checked: bool = False) -> str:
    """Compile and link; returns the path of the shared library (the checked one if `checked`)."""
    build_dir = BUILD + "_checked" if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    defs = ["-DLEAD_CHECKED=1"] if checked else []
    os.makedirs(build_dir, exist_ok=True)
    _write_jit_source(build_dir)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-I", INCLUDE, "-Xcompiler", "-fPIC", *defs]
    jobs = []
    for src in CU_SOURCES:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if ptxas_info:
            cmd.insert(1, "-Xptxas=-v")
        jobs.append((cmd, obj))
    for src in CPP_SOURCES:
        obj = os.path.join(build_dir, src.replace(".cpp", ".o"))
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", *defs, "-I", INCLUDE, "-I", build_dir,
               "-I", os.path.join(CUDA_HOME, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
        jobs.append((cmd, obj))
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        outs = list(ex.map(lambda j: _run(j[0]), jobs))
    if verbose or ptxas_info:
        for o in outs:
            if o.strip():
                print(o)
    tmp = lib + ".tmp"
    libdir = os.path.join(CUDA_HOME, "lib64")
    _run([nvcc, *ARCH, "-shared", "-o", tmp, *[o for _, o in jobs], "-L", libdir,
          "-lnvrtc", "-Xlinker", f"-rpath,{libdir}"])
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv, checked="--checked" in sys.argv))
