"""Host-side logic of bench.py (no GPU): the algorithmic-bytes model and the
rule that measured DRAM traffic is reported only for the kernel source and
first-step form it was captured on."""
import hashlib
import json
import os

import bench


def test_algorithmic_bytes_is_32T_68E_4C():
    # per sample: alias sector + header (64 B); per member: row sector + write
    # (36 B); per non-source member: source sector (32 B); per coin: threshold
    for T, E, C in ((1, 1, 0), (10, 41, 664), (10_000_000, 41_685_976, 664_326_661)):
        assert bench.algorithmic_bytes(T, E, C, True) == 32 * T + 68 * E + 4 * C
        assert bench.algorithmic_bytes(T, E, C, False) == 32 * T + 68 * E


def test_step_ids_partition_the_id_stream():
    # step i on rank r of N: block i N + r; blocks are disjoint and consecutive
    for world in (1, 2, 3, 8):
        firsts = [bench.step_first_id(i, r, world, 1000) for i in range(4) for r in range(world)]
        assert firsts == [1000 * b for b in range(4 * world)]


def test_alu_peak_derivation():
    # 152 SMs x 64 multiply-adds per clock / 40 per Philox block x 2.07 GHz
    assert abs(bench.alu_peak_blocks_per_s(152, 2070.0) - 503.424e9) < 1e3


def _fake_root(tmp_path, src: bytes, record: dict):
    os.makedirs(tmp_path / "profiles")
    os.makedirs(tmp_path / "paper_1709_03565_gb300" / "csrc")
    (tmp_path / "paper_1709_03565_gb300" / "csrc" / "sample.cu").write_bytes(src)
    (tmp_path / "profiles" / "iis_sampler_dram.json").write_text(json.dumps(record))


def test_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    src = b"// sampler source\n__global__ void k(int* a) { a[0] = 1; }\n"
    record = {"sample_cu_sha256": bench.code_sha(src), "first_step": "bucket",
              "dram_bytes_per_sample": 497.5, "workload_key": bench.C2_WORKLOAD}
    _fake_root(tmp_path, src, record)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic_per_sample("bucket") == 497.5
    assert bench._traffic_per_sample("rejection") is None  # captured on the other form
    (tmp_path / "paper_1709_03565_gb300" / "csrc" / "sample.cu").write_bytes(src + b"/* a comment\n edit */\n")
    assert bench._traffic_per_sample("bucket") == 497.5  # comments do not change the kernel
    (tmp_path / "paper_1709_03565_gb300" / "csrc" / "sample.cu").write_bytes(src.replace(b"= 1", b"= 2"))
    assert bench._traffic_per_sample("bucket") is None  # the kernel changed since the capture


def test_committed_record_names_its_capture():
    d = json.load(open(os.path.join(bench.ROOT, "profiles", "iis_sampler_dram.json")))
    assert d["first_step"] in ("bucket", "rejection")
    assert d["dram_bytes_per_sample"] > 0 and len(d["sample_cu_sha256"]) == 64
    assert d["command"].startswith("ncu ") and "--clock-control none" in d["command"]


def test_profile_summaries_name_commands_on_committed_files():
    """Every ncu summary gives the command that made it; the command runs
    ncu with --clock-control none on the committed bench or the package,
    nothing else."""
    pdir = os.path.join(bench.ROOT, "profiles")
    mds = [f for f in os.listdir(pdir) if f.endswith(".md")]
    assert mds
    for f in mds:
        blocks = open(os.path.join(pdir, f)).read().split("```")[1::2]  # fenced code blocks
        cmds = [ln.strip() for b in blocks for ln in b.splitlines() if ln.strip().startswith("ncu ")]
        assert cmds, f
        for c in cmds:
            assert "--clock-control none" in c, f
            assert (" python bench.py" in c or (" python -c " in c and "paper_1709_03565_gb300" in c)), f
            assert "_work" not in c, f
            if "--set" in c or "--section" in c:  # full captures: one kernel, a few launches
                k = c.split(" -k ", 1)[1].split()[0] if " -k " in c else ""
                assert k and "|" not in k, f
                assert " -c " in c and int(c.split(" -c ", 1)[1].split()[0]) <= 3, f
