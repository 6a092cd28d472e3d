"""Host-side pieces of bench.py that need no GPU: the kernel-source hash that
keys the stored DRAM-traffic record covers code only, so comment edits keep
the record and code edits drop it (the bench then reports traffic null)."""
import bench


def test_code_only_ignores_comments_and_blank_lines():
    a = "int f(int x) {\n  // one comment\n  return x + 1;  // trailing\n}\n\n/* block\n   comment */\n"
    b = "int f(int x) {\n  return x + 1;\n}\n"
    assert bench._code_only(a) == bench._code_only(b)


def test_code_only_sees_code_changes():
    a = "int f(int x) {\n  return x + 1;\n}\n"
    b = "int f(int x) {\n  return x + 2;\n}\n"
    assert bench._code_only(a) != bench._code_only(b)


def test_unknown_count_matches_the_oracle_meshes():
    """unique unknowns = nodes off the boundary: the 6-tet cube at level 8 has
    255^3; the 24- and 12-tet cubes agree with the oracle's level meshes."""
    from oracle import hhg_oracle as O
    from paper_1709_06793_gb300 import inputs as I
    _, T = I.kuhn_cube()
    assert bench.unknowns_of(T, 8) == 255 ** 3
    for mesh, levels in ((I.cube24, (1, 2, 3, 4)), (I.cube12, (1, 2, 3)), (I.cube48, (1, 2, 3)), (I.unit_tet, (2, 3))):
        V, T = mesh()
        for level in levels:
            lm = O.LevelMesh(O.MacroMesh(V, T), level)
            assert bench.unknowns_of(T, level) == len(lm.unknowns), (mesh.__name__, level)


def test_reference_arm_line_states_the_sample_it_timed(monkeypatch, capsys):
    """The reference arm times the oracle at its sample level on every host
    core and says so in its line (level, processes, cores)."""
    import json

    monkeypatch.setattr(bench, "CPU_LEVEL", 2)
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)

    class Args:
        gpus, steps, warmup = 1, 2, 1

    out = bench.run_reference(Args())
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line == json.loads(json.dumps(out))
    assert line["impl"] == "reference" and line["config"]["level"] == 2
    assert line["config"]["processes"] == line["cpu_baseline"]["cores"] == bench.host_info()["nproc"]
    assert "level 2" in line["config"]["workload"] and "level 9" not in line["config"]["workload"]
    assert line["value"] > 0 and line["e2e"]["value"] == line["value"]


def test_interface_copies_count_the_stored_face_nodes():
    """Stored nodes minus interior nodes, per tet: at level 1 every node of a
    tet is on its boundary; a tet at level 2 has one interior node."""
    from paper_1709_06793_gb300 import inputs as I
    _, T = I.cube24()
    assert bench.interface_copies(T, 1) == 24 * 10
    assert bench.interface_copies(T, 2) == 24 * (35 - 1)


def test_traffic_record_applies_only_to_its_kernel_and_sources(monkeypatch):
    """The stored counters scale per kernel unit while the sources hash to
    the recorded value and the recorded volume kernel runs; otherwise the
    bench reports no traffic."""
    rec = bench.NCU_TRAFFIC["bf16k_cube24"]
    monkeypatch.setattr(bench, "_kernel_sha", lambda: rec["sha"])
    t, src = bench._traffic("bf16k_cube24", 1000, 10, rec["vkernel"])
    assert abs(t - (rec["volume_bytes_per_node"] * 1000 + rec["interface_bytes_per_copy"] * 10)) < 1e-6 and src
    other = 1 if rec["vkernel"] != 1 else 2
    assert bench._traffic("bf16k_cube24", 1000, 10, other) == (None, None)
    monkeypatch.setattr(bench, "_kernel_sha", lambda: "0" * 16)
    assert bench._traffic("bf16k_cube24", 1000, 10, rec["vkernel"]) == (None, None)
