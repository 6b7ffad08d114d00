"""Host-side logic of bench.py that needs no GPU: the per-launch DRAM traffic lookup
(keyed by the hash of the kernel source, so counters taken on other code are never
reported) and the whole-job throughput arithmetic."""
import hashlib
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _tree(tmp_path, source_text, lines):
    csrc = tmp_path / "paper_1912_04582_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "tucker_kernels.cu").write_text(source_text)
    (csrc / "full_kernels.cu").write_text("full " + source_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.txt").write_text("\n".join(lines) + "\n")
    return tmp_path


def _h(text):
    return hashlib.sha256(text.encode()).hexdigest()[:16]


def test_traffic_is_read_for_the_current_source_only(tmp_path, monkeypatch):
    src = "// kernels, version A\n"
    root = _tree(tmp_path, src, [
        "# comment line tucker_eig 0000000000000000 1",
        f"tucker_eig {_h(src)} 54138965",
        "tucker_asm 0123456789abcdef 601009152",  # taken on other code
        f"full {_h('full ' + src)} 4362103000",
    ])
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench._traffic("tucker_eig") == 54138965.0
    assert bench._traffic("tucker_asm") is None
    assert bench._traffic("tucker_gram_mode1") is None
    assert bench._traffic("full") == 4362103000.0
    # any change to the kernel source invalidates its counters
    (root / "paper_1912_04582_gb300" / "csrc" / "tucker_kernels.cu").write_text(src + " ")
    assert bench._traffic("tucker_eig") is None


def test_traffic_without_the_file_is_null(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench._traffic("tucker_eig") is None


@pytest.mark.parametrize("world,steps,ms", [(1, 20, 61.5), (2, 20, 70.0), (8, 5, 12.0)])
def test_job_value_counts_every_rank(world, steps, ms):
    upd = 4096 * 32 ** 3
    v = bench.job_value(world, upd, steps, ms)
    assert v == pytest.approx(world * upd * steps / (ms / 1e3), rel=1e-12)


def test_assembly_terms_count_the_rank_one_terms_of_each_cell():
    """The GEMM-form assembly's work model: K = 4 Shakhov parts + 2 r1 for the cell + per
    face r1 of the neighbour or one ghost.  On a 4^3 cavity with every rank 2: corner cells
    (3 walls) 4 + 4 + 3*2 + 3 = 17, edge cells 18, face cells 19, interior cells 20, in the
    counts 8 / 24 / 24 / 8; with rank 1 in one interior cell its six neighbours lose 1."""
    import numpy as np
    import workloads as W
    wl = W.cavity(nside=4, N=8, seed=3)
    r = np.full(wl.n_cell, 2.0)
    K = bench.assembly_terms(wl, r)
    assert sorted(np.unique(K).tolist()) == [17, 18, 19, 20]
    assert [int((K == v).sum()) for v in (17, 18, 19, 20)] == [8, 24, 24, 8]
    ijk = np.asarray(wl.cell_ijk)
    c = int(np.flatnonzero((ijk == [1, 1, 1]).all(axis=1))[0])
    r2 = r.copy()
    r2[c] = 1.0
    d = K - bench.assembly_terms(wl, r2)
    assert d[c] == 2  # its own 2 r1
    nb = [int(np.flatnonzero((ijk == ijk[c] + e).all(axis=1))[0])
          for e in np.vstack([np.eye(3, dtype=int), -np.eye(3, dtype=int)])]
    assert all(d[q] == 1 for q in nb) and d.sum() == 2 + 6


@pytest.mark.parametrize("N,tc", [((48, 48, 48), True), ((64, 64, 64), True),
                                  ((32, 24, 20), True), ((40, 13, 7), False),
                                  ((72, 16, 16), False)])
def test_gram_on_tensor_cores_follows_the_library_rule(N, tc):
    """N1 <= 64 and N2 N3 a multiple of 8 up to 4096 (64^3: N2 N3 = 4096 is allowed; 40 x 13 x
    7: 91 columns, not a multiple of 8; 72 first-mode rows: too many)."""
    assert bench.gram_on_tensor_cores(N) == tc


class _FakeEvent:
    def __init__(self, **kw):
        pass

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 100.0


class _FakeSolver:
    """Counts steps; its 'residual' shrinks with the steps taken."""

    def __init__(self, wl, **kw):
        self.n = 0
        self.h = self
        self.kw = kw

    def step(self, n=1, residual=True):
        self.n += n
        return 1.0 / (1 + self.n)

    def f(self):
        return self.n

    def close(self):
        pass


def test_lusgs_extra_reports_step_time_and_convergence(monkeypatch):
    """The implicit-step extra of the C2 configuration: step time against the explicit
    step, and both schemes' steady residual at the same step counts."""
    import types
    import torch
    monkeypatch.setattr(torch.cuda, "Event", _FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)
    made = []

    def solver(wl, **kw):
        s = _FakeSolver(wl, **kw)
        made.append(s)
        return s
    P = types.SimpleNamespace(Solver=solver,
                              api=types.SimpleNamespace(dvm_init_f=lambda h, f: None))
    NAT = types.SimpleNamespace(DVM_SCHEME_LUSGS=1)
    out = bench.run_lusgs(P, NAT, types.SimpleNamespace(cuda_stream=0), full_ms=7.0)
    assert "error" not in out
    assert out["ms_per_step"] == 10.0 and abs(out["vs_explicit_step"] - 10.0 / 7.0) < 1e-12
    hist = out["steady_residual_after_steps"]
    assert [k for k, _ in hist["explicit_cfl0.5"]] == [100, 200, 300]
    assert [k for k, _ in hist["lusgs_cfl20"]] == [100, 200, 300]
    lus = [s for s in made if s.kw.get("scheme") == 1]
    assert len(lus) == 1 and lus[0].n == 300 and lus[0].kw["cfl"] == 20.0


def test_lusgs_extra_survives_a_failure(monkeypatch):
    import types
    import torch
    monkeypatch.setattr(torch.cuda, "synchronize", lambda: None)

    def solver(wl, **kw):
        raise RuntimeError("no device")
    P = types.SimpleNamespace(Solver=solver, api=None)
    out = bench.run_lusgs(P, types.SimpleNamespace(DVM_SCHEME_LUSGS=1),
                          types.SimpleNamespace(cuda_stream=0), full_ms=7.0)
    assert out["error"].startswith("no device")


def test_cylinder_workload_options():
    wl = bench.make_workload("cylinder")
    assert wl.n_cell == 1606 and wl.N == (64, 64, 64)
    assert bench.make_workload("cylinder_ogrid").n_cell == 1600


class _FakeServer:
    def __init__(self, budget, slots):
        self.sub = []

    def submit(self, wl, **kw):
        self.sub.append(kw)
        return len(self.sub) - 1

    def run(self, seconds):
        return 0

    def poll(self, t):
        return {"state": 2 if t % 2 == 0 else 3, "steps": 100 + t, "residual": 1e-5,
                "latency_s": 0.5 + t}

    def error(self, t):
        return ""

    def close(self):
        pass


@pytest.mark.parametrize("implicit", [False, True])
def test_serving_mix_reports_converged_solves_only(monkeypatch, implicit):
    import types
    made = []

    def server(b, s):
        made.append(_FakeServer(b, s))
        return made[-1]
    monkeypatch.setattr(bench.time, "perf_counter",
                        iter(float(x) for x in range(10 ** 6)).__next__)
    P = types.SimpleNamespace(Server=server)
    out = bench.run_serving(P, n_req=6, implicit=implicit)
    assert out["requests"] == 6 and out["converged"] == 3 and out["not_converged"] == 3
    assert out["median_steps_to_converge"] == 102.0
    kw = made[0].sub
    assert len(kw) == 6
    if implicit:
        assert all(k["scheme"] == 1 and k["format"] == 0 and k["cfl"] == 20.0 for k in kw)
        assert "implicit LU-SGS" in out["mix"]
    else:
        assert all(k["format"] == 1 and "scheme" not in k for k in kw)
