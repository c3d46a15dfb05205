"""Host-side logic of bench.py, no GPU: the reference arm's JSON line (the
oracle on the host cores), the staleness rule of the committed ncu figures,
and the replica jobs of the parallel oracle timing."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--windows", "2"], capture_output=True, text=True, timeout=300,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_committed_counters_are_tied_to_their_sources(tmp_path, monkeypatch):
    import bench
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for tag, e in d.items():
        assert e["sources"] and e["command"].startswith("ncu ") and "--clock-control none" in e["command"]
        assert bench.load_traffic(tag) in (e["bytes_per_launch"], None), tag  # the figure, or null once stale
    # a figure whose sources changed reads as null
    fake = tmp_path / "profiles"
    fake.mkdir()
    e = dict(d["k_resident_batched"], source_sha256="0" * 64)
    (fake / "traffic.json").write_text(json.dumps({"k_resident_batched": e}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda names=None: "1" * 64)
    assert bench.load_traffic("k_resident_batched") is None


def test_oracle_jobs_cover_every_replica():
    import bench
    from paper_2004_09081_gb300 import workloads
    wl = workloads.batched_batio3(0)
    jobs = bench.oracle_jobs(wl, 0)
    assert [j["r"] for j in jobs] == list(range(len(wl.replicas)))
    for j, rep in zip(jobs, wl.replicas):
        assert j["cells"] == tuple(rep.cells) and j["n_vac"] == rep.n_vac and j["T"] == rep.T
        assert all(c % f == 0 or c // f >= 2 for c, f in zip(j["cells"], j["nf"]))
