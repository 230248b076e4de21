"""Host logic of bench.py that needs no GPU: the DRAM-traffic record is reported only for
the kernel sources and workload it was captured on, and the roofline peak falls back to
the stated figure when no measured peaks file exists."""
import json

import bench


def _record(path, sha, workload, nbytes):
    path.write_text("# traffic\n\n"
                    f"- kernel_sources_sha1: `{sha}`\n"
                    f"- workload: `{workload}`\n"
                    f"- dram_bytes_per_launch: {nbytes}\n")


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    rec = tmp_path / "traffic.md"
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(rec))
    assert bench.stage_traffic("pl_n1e8") is None  # no record
    _record(rec, bench.kernel_sources_sha1(), "pl_n1e8", 123456789)
    assert bench.stage_traffic("pl_n1e8") == 123456789
    assert bench.stage_traffic("pl_n1e7") is None  # another workload
    _record(rec, "0" * 40, "pl_n1e8", 123456789)
    assert bench.stage_traffic("pl_n1e8") is None  # captured on other sources
    _record(rec, bench.kernel_sources_sha1(), "pl_n1e8", "n/a")
    assert bench.stage_traffic("pl_n1e8") is None  # unreadable figure


def test_kernel_sources_hash_covers_every_sampler_source():
    import hashlib
    import os

    csrc = os.path.join(bench.ROOT, "paper_1406_1215_gb300", "csrc")
    h = hashlib.sha1()
    for f in bench.KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    assert bench.kernel_sources_sha1() == h.hexdigest()
    # every file of the kernel directory that the sampler's translation unit includes is
    # hashed (the public C header, outside it, declares the interface only)
    src = open(os.path.join(csrc, "sample.cu")).read()
    local = [ln.split('"')[1] for ln in src.splitlines() if ln.startswith('#include "')]
    seen, todo = set(), list(local)
    while todo:
        f = todo.pop()
        if f in seen:
            continue
        seen.add(f)
        for ln in open(os.path.join(csrc, f)).read().splitlines():
            if ln.startswith('#include "') and "/" not in ln.split('"')[1]:
                todo.append(ln.split('"')[1])
    assert seen <= set(bench.KERNEL_SOURCES), seen - set(bench.KERNEL_SOURCES)


def test_peaks_measured_or_fallback(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6762.3}))
    assert bench.peaks() == (6762.3, "measured")
