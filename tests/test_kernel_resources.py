"""Register and stack use of the hot kernels, from the compiler's resource report (ptxas -v).

The three-step 2D kernel once kept its nine stage values in local memory because a stored-stage
index known only at run time made the compiler index them dynamically; nothing in its results
showed it, only its speed (12% of the time per launch).  These checks fail when such a stack frame
comes back, or when the kernel no longer fits the resident CTAs per SM it is launched for.  They
compile on the CPU (nvcc cross-compiles for sm_103a) and need no GPU."""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_0906_5170_gb300", "csrc")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def _resources(source, tmp_path):
    """{kernel mangled name: (stack frame bytes, spill store bytes, registers)} of one source."""
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    out = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
                          "-I", CSRC, "-I", os.path.join(ROOT, "include"), "-Xptxas", "-v", "-c",
                          os.path.join(CSRC, source), "-o", str(tmp_path / "k.o")],
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    res, cur, frame = {}, None, None
    for line in out.stderr.splitlines():
        m = re.search(r"Compiling entry function '(\S+)'", line)
        if m:
            cur = m.group(1)
        m = re.search(r"(\d+) bytes stack frame, (\d+) bytes spill stores", line)
        if m:
            frame = (int(m.group(1)), int(m.group(2)))
        m = re.search(r"Used (\d+) registers", line)
        if m and cur:
            res[cur] = (frame[0], frame[1], int(m.group(1)))
    assert res, out.stderr[-2000:]
    return res


def test_three_step_kernel_keeps_its_stage_values_in_registers(tmp_path):
    res = _resources("step2d_tk.cu", tmp_path)
    fp32 = {k: v for k, v in res.items() if "k_step2d_tkIf" in k}
    assert len(fp32) == 1, list(res)
    frame, spill, regs = next(iter(fp32.values()))
    assert frame == 0 and spill == 0, f"stack frame {frame} B, spill {spill} B"
    assert regs <= 64, f"{regs} registers: eight CTAs of 128 threads per SM no longer fit"


def test_two_step_march_variants_do_not_spill(tmp_path):
    res = _resources("step6m2.cu", tmp_path)
    mar2 = {k: v for k, v in res.items() if "k_mar2" in k}
    assert len(mar2) == 8, list(res)
    bad = {k: v for k, v in mar2.items() if v[0] or v[1]}
    assert not bad, bad
