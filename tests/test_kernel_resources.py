"""Register budget of the hot FP32 stage kernel, checked at build time (no
GPU): the Euler / LP / Rusanov stage kernel of p = 3, in the two
instantiations that large grids take (plain and low-part prefetch), must fit
the 64 registers that let four 256-thread CTAs share an SM, without spilling;
the one for grids of at most two CTAs per SM must not spill either.  A regression here costs a
quarter of the resident warps or adds local-memory traffic to every launch.
The figures come from ptxas's resource report (-Xptxas -v)."""
import functools
import os
import re
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1709_01619_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


@functools.lru_cache(maxsize=None)
def ptxas_report(src):
    """{entry: {"regs": n, "spill": bytes}} of one translation unit."""
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as tmp:
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c", os.path.join(CSRC, src),
               "-o", os.path.join(tmp, "k.o")]
        r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    report, current = {}, None
    for line in r.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            current = m.group(1)
            report[current] = {}
            continue
        if current is None:
            continue
        m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
        if m:
            report[current]["spill"] = int(m.group(1)) + int(m.group(2))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            report[current]["regs"] = int(m.group(1))
    return report


def test_p3_fp32_stage_kernel_fits_four_ctas_without_spills():
    report = ptxas_report("cpr_stage_f32_p3.cu")
    # cpr_stage_kernel<float, 3, EULER, DIV_LP, FLUX_RUSANOV, 8, 8, false, PF, WIDE>
    pre = "_ZN3cpr16cpr_stage_kernelIfLi3ELi1ELi0ELi0ELi8ELi8ELb0E"
    hot = {k[len(pre):len(pre) + 12]: report[k] for k in report if k.startswith(pre)}
    assert sorted(hot) == ["Lb0ELb0EEEvN", "Lb0ELb1EEEvN", "Lb1ELb0EEEvN"], sorted(report)
    for variant in ("Lb0ELb0EEEvN", "Lb1ELb0EEEvN"):  # plain, low-part prefetch
        assert hot[variant]["regs"] <= 64, (variant, hot[variant])
        assert hot[variant]["spill"] == 0, (variant, hot[variant])
    # the instantiation for grids of at most two CTAs per SM: 256 threads,
    # two CTAs, so up to 128 registers, and no spills
    wide = hot["Lb0ELb1EEEvN"]
    assert wide["regs"] <= 128 and wide["spill"] == 0, wide


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_two_cta_instantiations_do_not_spill(p):
    """The FP32 Euler stage kernels compiled for grids of at most two CTAs per
    SM (every divergence and flux) exist for every order and keep all their
    state in registers."""
    report = ptxas_report(f"cpr_stage_f32_p{p}.cu")
    pre = f"_ZN3cpr16cpr_stage_kernelIfLi{p}ELi1E"
    wide = {k: v for k, v in report.items() if k.startswith(pre) and k.endswith("Lb0ELb0ELb1EEEvNS_9StageArgsIT_EE")}
    assert len(wide) == 4, sorted(report)  # LP / chain rule x Rusanov / Roe
    for k, v in wide.items():
        assert v["spill"] == 0, (k, v)
