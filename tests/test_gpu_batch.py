"""Batched solves (yy_batch_*): many fields of uneven shape in one CUDA graph.

Checks, per the batched workload's test plan:
  - every field of a batch equals the same field solved alone (float64,
    bitwise: the graph runs the same kernels on the same data), and the
    grouped solves (one launch per stage over all fields, tensor-core forms)
    equal the per-field graphs and the fields solved alone bitwise;
  - graph replay is bitwise deterministic, and new buffers are recorded anew;
  - the 64-field workload (n_r ~ U{100..600}, 2 / 1.5 / 1 degree cells,
    l_max ~ U{10..40}) in the tuned FP16X2 form agrees with the float64 GPU
    path field by field within the form's tolerance (Phi 1e-6 pointwise,
    -grad Phi 1e-5 normwise) and with the float64 oracle on sampled cells.
"""

import numpy as np
import pytest

from paper_1806_04593_gb300 import inputs

from .gpu_common import field_err, grad_err, lib, phi_err, require_gpu

pytestmark = pytest.mark.gpu

# FP16X2 against the float64 path over the 64 uneven fields (l_max up to 40):
# Phi pointwise at the 1e-6 target (worst measured 3.8e-7), -grad Phi
# normwise at 4x the worst measured (2.5e-6)
TOL_PHI, TOL_GRAD = 1e-6, 1e-5


@pytest.fixture(scope="module")
def yy():
    require_gpu()
    return lib()


def _small_specs():
    return [
        inputs.tiny_grid(),
        inputs.GridSpec("b1", np.logspace(-3, 0, 61), 45, 135, 0.0, 0.0, 10),
        inputs.GridSpec("b2", np.logspace(-4, 0, 41), 60, 180, 0.0, 0.0, 12),
        inputs.GridSpec("b3", np.concatenate([[0.0], np.logspace(-2, 0, 37)]), 20, 57, 0.03, 0.05, 7),
    ]


def _fields(specs, dev, gradient=True, seed0=5):
    import torch
    rho, out = [], []
    for f, sp in enumerate(specs):
        ry, rg = inputs.pns_density(sp, seed0 + f, 0.05)
        rho.append((torch.from_numpy(ry).to(dev), torch.from_numpy(rg).to(dev)))
        shape = (sp.n_r, sp.n_theta, sp.n_phi)
        o = [torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
        if gradient:
            o += [torch.empty((3,) + shape, dtype=torch.float64, device=dev) for _ in range(2)]
        out.append(o)
    return rho, out


def _run(b, rho, out, prec, stream=None):
    grad = len(out[0]) == 4
    b.potential([r[0] for r in rho], [r[1] for r in rho], [o[0] for o in out], [o[1] for o in out],
                [o[2] for o in out] if grad else None, [o[3] for o in out] if grad else None,
                prec=prec, stream=stream)


def test_batch_fp64_equals_fields_solved_alone(yy):
    import torch
    dev = torch.device("cuda", 0)
    specs = _small_specs()
    b = yy.Batch(specs)
    rho, out = _fields(specs, dev)
    _run(b, rho, out, "fp64")
    torch.cuda.synchronize()
    assert b.device_status() == yy.YY_OK
    assert b.launch_count() > 0
    for sp, r, o in zip(specs, rho, out):
        g = yy.Grid.from_spec(sp)
        ref = g.solve(r[0], r[1], gradient=True, prec="fp64")
        torch.cuda.synchronize()
        assert torch.equal(o[0], ref["phi_yin"]) and torch.equal(o[1], ref["phi_yang"]), sp.name
        assert torch.equal(o[2], ref["grad_yin"]) and torch.equal(o[3], ref["grad_yang"]), sp.name
        g.close()
    b.close()


def test_batch_grouped_equals_per_field_graphs_and_fields_alone(yy):
    """Grouped solves (one launch per stage over every field) give, in each
    tensor-core form, the results of the per-field graph and of each field
    solved alone bit for bit: each field keeps its own tiles, K segments and
    arithmetic.  The small batch has all three density row forms (rows of at
    most 2,048 cells, longer odd and longer even rows): eight kernels."""
    import torch
    dev = torch.device("cuda", 0)
    specs = _small_specs()
    for prec in ("fp16x2", "bf16x3", "tf32"):
        b = yy.Batch(specs)
        b.prepare(prec)
        b.set_grouping(1)                             # one group: every stage one launch
        rho, grouped = _fields(specs, dev)
        _run(b, rho, grouped, prec)
        torch.cuda.synchronize()
        assert b.device_status() == yy.YY_OK
        assert b.launch_count() == 8, (prec, b.launch_count())
        b.set_grouping(2)                             # two groups side by side: the same results
        _, two = _fields(specs, dev)
        _run(b, rho, two, prec)
        torch.cuda.synchronize()
        assert 12 <= b.launch_count() <= 16, (prec, b.launch_count())
        for x, y in zip(grouped, two):
            for a, c in zip(x, y):
                assert torch.equal(a, c), prec
        b.set_grouping(0)
        _, per_field = _fields(specs, dev)
        _run(b, rho, per_field, prec)
        torch.cuda.synchronize()
        assert b.launch_count() > 8 * len(specs) // 2
        for sp, r, x, y in zip(specs, rho, grouped, per_field):
            for a, c in zip(x, y):
                assert torch.equal(a, c), (prec, sp.name)
            g = yy.Grid.from_spec(sp)
            g.prepare(prec)
            alone = g.solve(r[0], r[1], gradient=True, prec=prec)
            torch.cuda.synchronize()
            for key, a in zip(("phi_yin", "phi_yang", "grad_yin", "grad_yang"), x):
                assert torch.equal(a, alone[key]), (prec, sp.name, key)
            g.close()
        b.close()


def test_batch_graph_replay_is_deterministic_and_rebinds(yy):
    import torch
    dev = torch.device("cuda", 0)
    specs = _small_specs()
    b = yy.Batch(specs)
    b.prepare("fp16x2")
    rho, out = _fields(specs, dev)
    _run(b, rho, out, "fp16x2")
    first = [[t.clone() for t in o] for o in out]
    for o in out:
        for t in o:
            t.fill_(float("nan"))
    _run(b, rho, out, "fp16x2")                       # replay of the cached graph
    torch.cuda.synchronize()
    for a, o in zip(first, out):
        for x, y in zip(a, o):
            assert torch.equal(x, y)
    _, out2 = _fields(specs, dev)                     # other output buffers: recorded anew
    _run(b, rho, out2, "fp16x2")
    torch.cuda.synchronize()
    for a, o in zip(first, out2):
        for x, y in zip(a, o):
            assert torch.equal(x, y)
    assert b.device_status() == yy.YY_OK
    b.close()


def test_batched_workload_tuned_fp16x2(yy, oracle_grid):
    """The 64-field workload: tuned FP16X2 batch against the float64 GPU path
    (every field, whole fields) and against the oracle (four fields, sampled
    cells)."""
    import torch
    dev = torch.device("cuda", 0)
    items = inputs.batched_specs()
    specs = [sp for sp, _, _ in items]
    b = yy.Batch(specs)
    chosen = b.tune("fp16x2", gradient=True, reps=1)
    assert len(chosen) == len(specs) and set(chosen) <= {yy.YY_ANALYSIS_DENSE, yy.YY_ANALYSIS_SEPARABLE}
    rho, out = [], []
    for sp, seed, eps in items:
        ry, rg = inputs.pns_density(sp, seed, eps)
        rho.append((torch.from_numpy(ry).to(dev), torch.from_numpy(rg).to(dev)))
        shape = (sp.n_r, sp.n_theta, sp.n_phi)
        out.append([torch.empty(shape, dtype=torch.float64, device=dev) for _ in range(2)]
                   + [torch.empty((3,) + shape, dtype=torch.float64, device=dev) for _ in range(2)])
    _run(b, rho, out, "fp16x2")
    torch.cuda.synchronize()
    assert b.device_status() == yy.YY_OK
    rng = np.random.default_rng(7)
    for f, (sp, r, o) in enumerate(zip(specs, rho, out)):
        g = yy.Grid.from_spec(sp)
        ref = g.solve(r[0], r[1], gradient=True, prec="fp64")
        torch.cuda.synchronize()
        for q, (phi, grad) in enumerate((("phi_yin", "grad_yin"), ("phi_yang", "grad_yang"))):
            assert phi_err(o[q].cpu().numpy(), ref[phi].cpu().numpy()) <= TOL_PHI, (f, phi)
            assert grad_err(o[2 + q].cpu().numpy(), ref[grad].cpu().numpy()) <= TOL_GRAD, (f, grad)
        g.close()
        if f % 16 == 0:
            cells = np.sort(rng.choice(sp.n_ang, 12, replace=False))
            ref_o = oracle_grid(sp).solve(r[0].cpu().numpy(), r[1].cpu().numpy(), gradient=True, cells=cells)
            j, k = np.divmod(cells, sp.n_phi)
            assert phi_err(o[0].cpu().numpy()[:, j, k], ref_o["phi_yin"]) <= TOL_PHI, f
            assert grad_err(o[3].cpu().numpy()[:, :, j, k], ref_o["grad_yang"]) <= TOL_GRAD, f
        del ref
    b.close()


def test_batch_fp64_ozaki_tuned_matches_fp64(yy):
    """The float64 results by the Ozaki scheme through the batch: tuned,
    captured in one graph, every field within 2e-13 of the float64 batch and
    bitwise equal to the same field solved alone with the evaluation the
    tuner picked for it."""
    import torch
    dev = torch.device("cuda", 0)
    specs = _small_specs()
    b = yy.Batch(specs)
    chosen = b.tune("fp64_ozaki", gradient=True, reps=1)
    rho, out = _fields(specs, dev)
    _, ref = _fields(specs, dev)
    _run(b, rho, out, "fp64_ozaki")
    _run(b, rho, ref, "fp64")
    torch.cuda.synchronize()
    assert b.device_status() == yy.YY_OK
    for sp, o, r in zip(specs, out, ref):
        for key, x, y in zip(("phi_yin", "phi_yang", "grad_yin", "grad_yang"), o, r):
            assert field_err(key, x.cpu().numpy(), y.cpu().numpy()) <= 2e-13, (sp.name, key)
    names = {yy.ANALYSES[k]: k for k in yy.ANALYSES}
    for f in (0, 3):
        g = yy.Grid.from_spec(specs[f])
        g.prepare("fp64_ozaki")
        g.set_analysis(names[chosen[f]])
        alone = g.solve(rho[f][0], rho[f][1], gradient=True, prec="fp64_ozaki")
        torch.cuda.synchronize()
        assert torch.equal(alone["phi_yin"], out[f][0]) and torch.equal(alone["grad_yang"], out[f][3]), f
        g.close()
    b.close()
