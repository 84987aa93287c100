"""Builds the sm_103a shared library ``libmonc_proj.so`` in-tree with nvcc."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmonc_proj.so")
# (source, extra defines, object name): kern_f32_ext.cu is compiled once per
# group of extended FP32 lengths and part (rows / columns)
SOURCES = [(f, [], os.path.splitext(f)[0]) for f in
           ("monc_proj.cu", "kern_f32_rows.cu", "kern_f32_cols.cu", "kern_f32_fused.cu", "kern_f64.cu",
            "kern_f32_refined.cu", "kern_krylov.cu", "kern_f32_pipe.cu", "kern_f32_tc.cu", "kern_f32_group.cu")]
SOURCES += [("kern_f32_ext.cu", [f"-DMP_EXT_GROUP={g}", f"-DMP_EXT_PART={part}"], f"kern_f32_ext{g}_{part}")
            for g in (1, 2, 3, 4) for part in (0, 1)]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return os.path.join(cand, "bin", "nvcc")
    found = shutil.which("nvcc")
    if not found:
        raise RuntimeError("nvcc not found")
    return found


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "monc_proj.h"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit in parallel, then link the shared library."""
    if not force and up_to_date():
        return LIB
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    common = [nvcc_path(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-I", os.path.join(ROOT, "include")]
    if verbose:
        common.append("-Xptxas=-v")
    common += os.environ.get("MONC_PROJ_NVCC_EXTRA", "").split()
    procs = []
    objs = []
    for src, defs, name in SOURCES:
        obj = os.path.join(objdir, name + ".o")
        objs.append(obj)
        procs.append((name, subprocess.Popen(common + defs + ["-c", os.path.join(CSRC, src), "-o", obj],
                                             stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    errors = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errors.append(f"{src}:\n{out}")
        elif verbose:
            print(out)
    if errors:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
    link = [nvcc_path(), *ARCH, "-shared", "-o", LIB + ".tmp"] + objs
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stdout + r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
