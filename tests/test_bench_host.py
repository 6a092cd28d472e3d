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
