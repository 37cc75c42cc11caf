"""Register budgets of the chain kernel, as the compiler reports them (CPU only:
nvcc cross-compiles one map format's translation unit with ptxas's verbose
output).  The autotuner and the bench name the launch configurations by these
budgets -- 128, 96, 80, 72 registers for one atom per lane, 128 and 96 for two
atoms per lane and for mixed tiles -- so every kernel must use exactly its
budget, and the budgets meant to run without spills must have none."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2303_09916_gb300", "csrc")

# (variant, tiles) -> registers; tiles 1 = one atom per lane, 2 = two, 3 = mixed
BUDGET = {(0, 1): 128, (1, 1): 96, (2, 1): 80, (3, 1): 72, (0, 2): 128, (1, 2): 96, (0, 3): 128, (1, 3): 96}
NO_SPILLS = {(0, 1), (1, 1), (0, 2), (0, 3), (1, 3)}


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def _report(stderr, fmt):
    found, entry = {}, None
    for line in stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            k = re.search(r"dock_chains_kernelILi%dELi(\d)ELi(\d)E" % fmt, m.group(1))
            entry = (int(k.group(1)), int(k.group(2))) if k else None
            continue
        if entry is None:
            continue
        m = re.search(r"(\d+) bytes spill stores", line)
        if m:
            found.setdefault(entry, {})["spill"] = int(m.group(1))
        m = re.search(r"Used (\d+) registers", line)
        if m:
            found.setdefault(entry, {})["regs"] = int(m.group(1))
    return found


@pytest.mark.slow
def test_chain_kernel_register_budgets(tmp_path):
    """Every map format's translation unit (FP32 / BF16 / FP16 maps, Eq. 4 and
    Eq. 3), compiled in parallel."""
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    procs = {}
    for fmt in range(6):
        cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-Xptxas", "-v",
               "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-c", os.path.join(CSRC, f"dock_fmt{fmt}.cu"),
               "-o", str(tmp_path / f"dock_fmt{fmt}.o")]
        procs[fmt] = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    for fmt, proc in procs.items():
        _, err = proc.communicate(timeout=900)
        assert proc.returncode == 0, err[-2000:]
        found = _report(err, fmt)
        assert set(found) == set(BUDGET), (fmt, sorted(found))
        for key, regs in BUDGET.items():
            assert found[key]["regs"] == regs, (fmt, key, found[key])
            if key in NO_SPILLS:
                assert found[key]["spill"] == 0, (fmt, key, found[key])
