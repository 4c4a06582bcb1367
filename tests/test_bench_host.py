"""Host logic of bench.py (no GPU): the paper's throughput used for vs_baseline, the parser of
the committed full-size ncu summary and its source check, the workload description and the
partition of marker blocks over replicas."""
import hashlib
import os

import bench
import synth


def test_paper_rate_is_the_section_3_1_figure():
    w = synth.WORKLOADS["n23000_m8900000_p20480_c20_u8"]
    assert abs(bench._paper_rate(w) - 8.9e6 * 20480 / 1108.0) < 1.0
    w2 = synth.WORKLOADS["n23000_m1000000_p2048_c10_2bit"]
    assert abs(bench._paper_rate(w2) - 8.9e6 * 2048 / 940.0) < 1.0
    assert bench._paper_rate(synth.WORKLOADS["n2000_m10000_p16_c5_2bit"]) is None  # N=2,000
    assert bench._paper_rate(synth.WORKLOADS["n23000_m500000_12panels_p8192_2bit"]) is None


def _fake_repo(tmp_path, sha):
    csrc = tmp_path / "paper_2604_21095_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k_tc2.cu").write_bytes(b"kernel a")
    (csrc / "tc_common.cuh").write_bytes(b"header b")
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / bench.PROFILE_TRAFFIC).write_text(
        "# title: with a colon\n\n| metric | value |\n|---|---|\n| a: b | c |\n\n"
        "Workload: something\n"
        "dram_bytes_per_launch: 123456\n"
        "tensor_pipe_active_pct: 91.20\n"
        f"source_sha256: {sha}\n"
        "Reading. text with a colon: here\n")
    return str(tmp_path)


def test_kernel_profile_needs_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    good = hashlib.sha256(b"kernel a" + b"header b").hexdigest()
    monkeypatch.setattr(bench, "ROOT", _fake_repo(tmp_path / "a", good))
    assert bench._kernel_profile() == {"dram_bytes_per_launch": 123456, "tensor_pipe_active": 0.912}
    monkeypatch.setattr(bench, "ROOT", _fake_repo(tmp_path / "b", "0" * 64))
    assert bench._kernel_profile() == {}
    monkeypatch.setattr(bench, "ROOT", str(tmp_path / "missing"))
    assert bench._kernel_profile() == {}


def test_committed_profile_parses():
    rec = {}
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", bench.PROFILE_TRAFFIC)
    for line in open(path):
        if ":" in line and not line.startswith(("|", "#", " ")):
            k, v = line.split(":", 1)
            rec[k.strip()] = v.strip()
    assert int(rec["dram_bytes_per_launch"]) > 4.9e9  # at least the compulsory operand bytes
    assert 0.0 < float(rec["tensor_pipe_active_pct"]) <= 100.0
    assert len(rec["source_sha256"]) == 64


def test_config_names_the_workload_and_its_l2_relation():
    w = synth.WORKLOADS["n23000_m8900000_p20480_c20_u8"]
    cfg = bench._config(w)
    assert cfg["workload"].startswith("n23000_m8900000_p20480_c20_u8")
    assert (cfg["N"], cfg["P"], cfg["C"]) == (23000, 20480, 20)
    assert "larger than L2" in cfg["l2"]


def test_replicas_partition_the_blocks():
    for ws in (1, 2, 3, 8):
        got = sorted(b for r in range(ws) for b in bench.rank_blocks(r, ws, 5))
        assert got == list(range(5 * ws))


def test_fused_joint_rule_and_bytes():
    """The bench counts the bytes of the path the library takes: the fused joint pass (the
    packed rows read twice) for small panels on blocks of at least one 128-marker tile per SM,
    else the decoded operand written and read per pass."""
    import bench
    assert bench.fused_joint(65536, 16, 20, 152) and bench.fused_joint(65536, 109, 20, 152)
    assert not bench.fused_joint(65536, 110, 20, 152)   # P + q - 1 = 129 > 128
    assert not bench.fused_joint(10000, 16, 5, 152)     # fewer 128-marker tiles than SMs
    assert not bench.fused_joint(65536, 16, 1, 152)     # no covariate projection
    N, M = 23000, 65536
    fused = bench._hbm_bytes_per_block(N, M, "u8", 16, 20, True)
    assert fused == 2 * M * N + 2 * 2 * 64 * 23040
    plain = bench._hbm_bytes_per_block(N, M, "u8", 16, 20, False)
    assert plain == M * N + 2 * (2 * M * 23040) + 2 * 2 * 16 * 23040
    two_pass = bench._hbm_bytes_per_block(N, M, "2bit", 300, 20, False)
    assert two_pass == M * 5750 + 3 * (2 * M * 23040) + 2 * 2 * 300 * 23040
    # dosage rows on 256-marker tiles: the joint pass writes the statistics, one read of the rows
    assert bench.one_pass_joint(N, M, "u8", 152) and not bench.one_pass_joint(N, M, "2bit", 152)
    assert not bench.one_pass_joint(N, 38_000, "u8", 152)   # fewer 256-marker tiles than SMs
    assert not bench.one_pass_joint(70_000, M, "u8", 152)   # sums of squares past 32 bits
    one = bench._hbm_bytes_per_block(N, M, "u8", 16, 20, True, True)
    assert one == M * N + 2 * 2 * 64 * 23040


def test_fused_projection_rule_and_bytes():
    """A panel too large for the joint pass (P + q - 1 > 128) takes the projection pass that
    writes the operand on blocks of at least one 128-marker tile per SM (with a 256-row joint
    operand, only where that pass writes the statistics): the bench counts the
    packed rows (once with the one-pass statistics, else twice), the 64 projection rows of hi +
    lo, the operand written once and read once, and the panel."""
    import bench
    N, M = 23000, 65536
    fp = bench.fused_projection
    assert fp(N, M, "u8", 110, 20, 152) and fp(N, M, "u8", 20480, 20, 152)
    assert fp(N, M, "2bit", 238, 20, 152)                  # P + q - 1 = 257: no joint operand
    assert not fp(N, M, "2bit", 237, 20, 152)              # the 256-row joint pass, counted rows
    assert not fp(N, 38_000, "u8", 200, 20, 152)           # the same on 128-marker tiles
    assert not fp(N, M, "u8", 109, 20, 152)                # the joint pass takes it
    assert not fp(N, 10000, "u8", 300, 5, 152)             # fewer 128-marker tiles than SMs
    assert not fp(N, M, "u8", 300, 1, 152)                 # no covariate projection
    op = bench._hbm_bytes_per_block(N, M, "u8", 300, 20, False, True, True)
    assert op == M * N + 2 * 2 * 64 * 23040 + 2 * (2 * M * 23040) + 2 * 2 * 300 * 23040
    tp = bench._hbm_bytes_per_block(N, M, "2bit", 300, 20, False, False, True)
    assert tp == 2 * M * 5750 + 2 * 2 * 64 * 23040 + 2 * (2 * M * 23040) + 2 * 2 * 300 * 23040
    # one read of the operand fewer than the decoded-operand path's, for an extra read of the
    # packed rows at most
    plain = bench._hbm_bytes_per_block(N, M, "2bit", 300, 20, False)
    assert plain - tp == 2 * M * 23040 - M * 5750 - 2 * 2 * 64 * 23040
