"""The reference arm of bench.py (the CPU oracle timed as it stands) prints one JSON line with
every key the benchmark contract asks for.  Runs on CPU in about 15 s."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_complete_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    j = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in j, key
    assert j["impl"] == "reference" and j["value"] > 0 and j["higher_is_better"] is True
    assert j["steps"] == 1 and j["warmup"] == 1 and j["dtype"] == "f64" and j["data"] == "synthetic"
    assert "workload" in j["config"]
    cb = j["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == j["value"] and cb["sample"]
    e = j["e2e"]
    assert e["value"] == j["value"] and e["unit"] == j["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def _bench():
    sys.path.insert(0, ROOT)
    import bench
    return bench


class _Info:
    """The gksl_info fields the bench's accounting reads, at the N = 1000 dimer's values."""
    nnz_q0, nnz_q1, D, long_rows, tail_nnz, ell_width_q0 = 18449538, 999000, 999999, 994, 512396, 18
    compact_escaped_rows, q1_folded = 2647, 1

    def __init__(self, variants, compact):
        self.rk4_variant, self.rk4_compact = variants, compact


def test_stage_accounting_at_n1000():
    """Algorithmic bytes and FP64 operations per stage launch at N = 1000, worked out by hand from
    their definitions (12 B per stored entry + 8 B of folded Q1 value per row + 17 vector passes
    of 8 B per step, averaged over 4 stages; 16-bit columns: 2 B less per entry, 2 B more per entry
    read with a 32-bit column; FP32: 4-byte values and the FP64 master update)."""
    b = _bench()
    nnz0, nnz1, D = _Info.nnz_q0, _Info.nnz_q1, _Info.D
    assert b.stage_bytes(nnz0, nnz1, D, 64, True) == 263394414
    assert b.stage_bytes(nnz0, nnz1, D, 64, False) == 267382422
    wide = _Info.tail_nnz + _Info.compact_escaped_rows * _Info.ell_width_q0
    assert b.stage_bytes(nnz0, nnz1, D, 64, True, wide) == 227615422
    assert b.stage_bytes(nnz0, nnz1, D, 32, True, wide) == 136817287
    assert b.stage_bytes(nnz0, nnz1, D, 32, True) == 172596279
    assert b.stage_fp64_ops(nnz0, D, _Info.long_rows, True) == 21516621.25
    assert abs(b.fp64_peak_gops(2070.0) - 629.28) < 1e-9
    info = _Info([0, 0], [0, 1])
    assert b.wide_entries(info, 0) is None and b.wide_entries(info, 1) == wide
    assert b.kernel_name(info, 0) == "k_stage64<S,18,true,false>"
    assert b.kernel_name(info, 1) == "k_stage32<S,18,true,true>"
    assert b.kernel_name(_Info([3, 2], [1, 0]), 0) == "k_stage_pdl<S,18,double,true,true>"
    assert b.kernel_name(_Info([3, 2], [1, 0]), 1) == "k_stage_r2<S,18,float,true>"


def test_source_hash_ignores_comments():
    b = _bench()
    code = "int f(int x) {\n    return x + 1;   // one more\n}\n/* block\n comment */\n"
    assert b.code_text(code) == b.code_text("int f(int x) { return x + 1; }")
    assert b.code_text(code) != b.code_text("int f(int x) { return x + 2; }")


def test_reference_arm_under_two_ranks_prints_once():
    """Launched as the multi-GPU runs are (torch.distributed.run, two ranks), the reference arm
    runs on rank 0 alone: one JSON line with n_gpus = 2, and every rank exits 0."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
