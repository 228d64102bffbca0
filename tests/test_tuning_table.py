"""Host logic of the persistent tuning table (no GPU): keys, JSON round trip,
and that a recorded shape is installed instead of timed again."""
import pytest


@pytest.fixture(scope="module")
def deco():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2509_18612_gb300 as d
    return d


def test_tuning_table_times_once_then_installs(deco, tmp_path, monkeypatch):
    from paper_2509_18612_gb300 import tuning as T
    calls = {"autotune": [], "set": []}
    monkeypatch.setattr(T.L, "deco_graph_info", lambda g: (g["n"], g["nnz"], 0))
    monkeypatch.setattr(T, "_gpu_name", lambda: "GB300")

    def fake_autotune(g, C, precision, objective, momentum, probe_steps):
        calls["autotune"].append((g["n"], C, precision))
        return 0x20a402, 9.3

    monkeypatch.setattr(T.L, "deco_autotune", fake_autotune)
    monkeypatch.setattr(T.L, "deco_set_tuning", lambda g, C, p, k: calls["set"].append((g["n"], C, p, k)))
    path = str(tmp_path / "tuning.json")
    g800, g900 = {"n": 800, "nnz": 38460}, {"n": 900, "nnz": 1000}
    tt = T.TuningTable(path)
    assert tt.ensure(g800, 1024, deco.DECO_PREC_FP32) == 0x20a402
    assert tt.ensure(g800, 1024, deco.DECO_PREC_FP32) == 0x20a402   # second time: installed, not timed
    assert calls["autotune"] == [(800, 1024, deco.DECO_PREC_FP32)]
    assert calls["set"] == [(800, 1024, deco.DECO_PREC_FP32, 0x20a402)]
    tt.save()
    # a new process reads the table back; other shapes are timed afresh
    tt2 = T.TuningTable(path)
    assert tt2.table == tt.table
    assert tt2.ensure(g800, 1024, deco.DECO_PREC_FP32) == 0x20a402
    tt2.ensure(g800, 2048, deco.DECO_PREC_FP32)
    tt2.ensure(g900, 1024, deco.DECO_PREC_FP32)
    tt2.ensure(g800, 1024, deco.DECO_PREC_BF16)
    assert len(calls["autotune"]) == 4
    assert T.shape_key(g800, 1024, deco.DECO_PREC_FP32) == "GB300|n=800|nnz=38460|w=0|C=1024|p=0"
