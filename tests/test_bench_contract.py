"""The bench's JSON line (CPU): the reference arm runs the FP64 oracle on
the host cores, so its line can be checked here without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_keeps_the_contract():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["unit"] == "sample-steps/s" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("rank2-fp32-K512-M256")


def test_roofline_traffic_comes_from_the_committed_profile():
    """The headline line's roofline `traffic` is read from the ncu summary of
    the kernels of the headline plan; each summary keeps the line the bench
    parses, equal to the read + write bytes of one full launch (the sum over
    both kernels of the split + companion pair)."""
    import re
    import bench
    cases = [("rank2_split_kernel<8>", "rank2_split_kernel_fp32_K512_M256_N10000.md"),
             ("rank2_split_kernel<8> + rank2_stream_kernel<8,4>",
              "rank2_split_and_stream_kernels_fp32_K512_M256_N10000.md")]
    for kname, fname in cases:
        t = bench.profiled_traffic(kname, 10000)
        assert isinstance(t, int) and t > 0
        text = open(os.path.join(ROOT, "profiles", fname)).read()
        rd = [int(x.replace(",", "")) for x in re.findall(r"dram__bytes_read\.sum \| ([\d,]+) B", text)]
        wr = [int(x.replace(",", "")) for x in re.findall(r"dram__bytes_write\.sum \| ([\d,]+) B", text)]
        if not rd:  # table with one row per kernel
            rows = re.findall(r"^\| rank2_\w+<[^|]*\| ([\d,]+) B \| ([\d,]+) B \|", text, re.M)
            rd = [int(a.replace(",", "")) for a, _ in rows]
            wr = [int(b.replace(",", "")) for _, b in rows]
        assert rd and t == sum(rd) + sum(wr), (fname, t, rd, wr)
        assert bench.profiled_traffic(kname, 1234) is None
