"""Learned quadrature orders: the order model's GPU kernels against the FP64
CPU reference (gradients, tensor-core inference), deterministic training, and
the learned near field judged by the oracle at high order, with the gain over
the fixed rule that meets the same error target."""
import numpy as np
import pytest

import mlp_ref
import synth
from parity_util import oracle_absolute, oracle_entries, rel_err_abs, sample_block_entries, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1510_07244_gb300 as pkg
    from paper_1510_07244_gb300 import order_model
    ctx = pkg.Context(0)
    yield pkg, ctx, order_model
    ctx.close()


def test_gradients_match_cpu_backprop(env):
    import torch
    pkg, ctx, _ = env
    mlp = ctx.bem_mlp_create(3)
    p, _ = ctx.bem_mlp_get_params(mlp)
    rng = np.random.default_rng(2)
    X = rng.normal(0, 1, (256, 8)).astype(np.float32)
    y = rng.integers(0, 6, 256).astype(np.int32)
    g = torch.zeros(ctx.bem_mlp_num_params(), dtype=torch.float32, device="cuda")
    loss = ctx.bem_mlp_gradients(mlp, to_dev(X, torch.float32), to_dev(y, torch.int32), g)
    ref_loss, ref_g = mlp_ref.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y)
    got = g.cpu().numpy().astype(np.float64)
    assert abs(loss - ref_loss) <= 1e-5 * abs(ref_loss)
    assert np.abs(got - ref_g).max() <= 1e-3 * np.abs(ref_g).max()
    big = np.abs(ref_g) > 1e-2 * np.abs(ref_g).max()
    assert np.all(np.abs(got[big] - ref_g[big]) <= 1e-3 * np.abs(ref_g[big]))
    ctx.bem_mlp_destroy(mlp)


def test_tensor_core_inference_matches_bf16_reference(env):
    import torch
    pkg, ctx, _ = env
    mlp = ctx.bem_mlp_create(5)
    p, _ = ctx.bem_mlp_get_params(mlp)
    rng = np.random.default_rng(4)
    n = 1000   # not a multiple of 16: ragged last tile
    X = rng.normal(0, 1, (n, 8)).astype(np.float32)
    logits = torch.zeros((n, 6), dtype=torch.float32, device="cuda")
    ctx.bem_mlp_infer(mlp, to_dev(X, torch.float32), logits)
    got = logits.cpu().numpy()
    ref = mlp_ref.forward(p.astype(np.float64), X, bf16=True)[-1]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 2e-2 * scale
    srt = np.sort(ref, axis=1)
    clear = srt[:, -1] - srt[:, -2] > 5e-2 * scale
    assert np.mean(np.argmax(got, 1)[clear] == np.argmax(ref, 1)[clear]) == 1.0
    ctx.bem_mlp_destroy(mlp)


def test_training_is_deterministic_and_learns(env):
    import torch
    pkg, ctx, om = env
    rng = np.random.default_rng(7)
    X = rng.normal(0, 1, (4000, 8)).astype(np.float32)
    y = np.clip((X[:, 0] + 2.5).astype(np.int32), 0, 5)      # a learnable rule
    Xd, yd = to_dev(X, torch.float32), to_dev(y, torch.int32)
    m1, l1 = om.fit(ctx, Xd, yd, epochs=12, batch=500, lr=1e-2, seed=11)
    m2, l2 = om.fit(ctx, Xd, yd, epochs=12, batch=500, lr=1e-2, seed=11)
    assert l1 == l2
    assert np.array_equal(ctx.bem_mlp_get_params(m1)[0], ctx.bem_mlp_get_params(m2)[0])
    assert l1[-1] < 0.3 * l1[0]
    ctx.bem_mlp_destroy(m1)
    ctx.bem_mlp_destroy(m2)


def _regular_pairs(mesh, bs_list, n, rng):
    out_a, out_b = [], []
    for bs in bs_list:
        r, c = bs.entry_indices()
        pick = rng.integers(min(n, len(r)), len(r))
        out_a.append(r[pick])
        out_b.append(c[pick])
    a = np.concatenate(out_a)
    b = np.concatenate(out_b)
    t = mesh.tris
    reg = ~np.array([len(set(t[i]) & set(t[j])) > 0 for i, j in zip(a, b)])
    return a[reg].astype(np.int32), b[reg].astype(np.int32)


KERNELS = [("laplace_dlp", 0.0), ("helmholtz_slp", 16.0)]


@pytest.fixture(scope="module")
def trained(env):
    """Order model trained on pairs of two small jittered octahedral spheres."""
    import torch
    pkg, ctx, om = env
    Xs, ys = [], []
    rng = synth.SplitMix64(151007244 + 5000)
    for n, s in ((16, 1), (24, 2)):
        mesh = synth.jitter(synth.octasphere(n), 0.05, 151007244 + 5000 + s)
        _, near, far = synth.workloads.h2_blocks(mesh, "p0", 32, 2.0, 16, s)
        mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
        a, b = _regular_pairs(mesh, (near, far), 12000, rng)
        ad, bd = to_dev(a, torch.int32), to_dev(b, torch.int32)
        for kernel, kappa in KERNELS:
            kd = pkg.kernel_desc(kernel, kappa)
            Xs.append(om.raw_features(ctx, mid, kd, ad, bd))
            ys.append(om.labels(ctx, mid, kd, ad, bd, tol=1e-7)[0])
        ctx.bem_mesh_free(mid)
    mlp, losses = om.fit(ctx, torch.cat(Xs), torch.cat(ys), epochs=40, batch=2048, lr=3e-3, seed=1)
    yield mlp, losses
    ctx.bem_mlp_destroy(mlp)


@pytest.mark.parametrize("precision", ["fp64", "mixed_full"])
@pytest.mark.parametrize("kernel,kappa", KERNELS)
def test_learned_near_field_meets_target_with_gain(env, trained, kernel, kappa, precision):
    """Held-out 8192-triangle jittered sphere: learned orders vs the oracle at
    Duffy order 10 (same singular rules) on whole sampled blocks, in the FP64
    form (one warp per pair) and the float form (one thread per pair for the
    classes whose rule is a product of a 2D rule)."""
    import torch
    pkg, ctx, om = env
    mlp, losses = trained
    assert losses[-1] < losses[0]
    ctx.bem_set_order_model(mlp, 0.95)
    mesh = synth.jitter(synth.octasphere(32), 0.05, 151007244 + 5099)
    _, near, _ = synth.workloads.h2_blocks(mesh, "p0", 32, 2.0, 16, 9)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    from parity_util import block_job
    q = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5,
             order_mode="learned", precision=precision)
    dt = torch.complex128 if kernel == "helmholtz_slp" else torch.float64
    out = torch.full((near.n_entries,), float("nan"), dtype=dt, device="cuda")
    ctx.bem_near_field([block_job(pkg, mid, near, kernel, kappa, q, out)])
    ctx.bem_sync()
    counts = ctx.bem_learned_counts()
    got_all = out.cpu().numpy()
    assert np.isfinite(got_all).all()
    pos = sample_block_entries(near, 10, synth.SplitMix64(3))
    r, c = near.entry_indices()
    qref = dict(q_regular=10, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
    ref = oracle_entries(mesh, "p0", r[pos], c[pos], kernel, kappa, qref)
    A = oracle_absolute(mesh, "p0", r[pos], c[pos], kernel, kappa, qref)
    err = rel_err_abs(got_all[pos], ref, A, r[pos]).max()
    assert err <= 1e-6, err
    # coupling blocks take learned orders too (no touching pairs there)
    _, _, far = synth.workloads.h2_blocks(mesh, "p0", 32, 2.0, 16, 9)
    outf = torch.full((far.n_entries,), float("nan"), dtype=dt, device="cuda")
    ctx.bem_coupling_blocks([block_job(pkg, mid, far, kernel, kappa, q, outf)])
    ctx.bem_sync()
    posf = sample_block_entries(far, 10, synth.SplitMix64(4))
    rf, cf = far.entry_indices()
    reff = oracle_entries(mesh, "p0", rf[posf], cf[posf], kernel, kappa, qref)
    Af = oracle_absolute(mesh, "p0", rf[posf], cf[posf], kernel, kappa, qref)
    errf = rel_err_abs(outf.cpu().numpy()[posf], reff, Af, rf[posf]).max()
    assert errf <= 1e-6, errf
    # gain: points per disjoint pair against the cheapest fixed rule meeting the
    # target on every pair of the training data (Duffy q=6: 1296 points)
    pts = np.dot(counts, pkg.ORDER_CLASS_POINTS) / max(1, sum(counts))
    assert pts < 0.25 * 1296, (counts, pts)
    print(f"learned {kernel}: class counts {counts}, {pts:.1f} points per disjoint pair, "
          f"max error {err:.2e} (target 1e-6)")
    ctx.bem_set_order_model(None, 0.0)
    ctx.bem_mesh_free(mid)


def test_learned_jobs_in_a_plan_equal_per_call_results(env, trained):
    """Learned-order jobs inside a plan (one CUDA graph with fixed-order jobs
    beside them) give the per-call learned results bit for bit, with the same
    class counts."""
    import torch
    from parity_util import block_job
    pkg, ctx, om = env
    mlp, _ = trained
    ctx.bem_set_order_model(mlp, 0.99)
    mesh = synth.jitter(synth.octasphere(24), 0.05, 151007244 + 5098)
    _, near, far = synth.workloads.h2_blocks(mesh, "p0", 32, 2.0, 16, 8)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    ql = dict(q_regular=3, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5,
              order_mode="learned", precision="mixed_full")
    qf = dict(ql, order_mode="fixed")
    res = {}
    for how in ("calls", "plan"):
        outs = {}
        jobs = {"near": [], "far": []}
        for kernel, kappa in KERNELS:
            dt = torch.complex128 if kernel == "helmholtz_slp" else torch.float64
            for nm, bs in (("near", near), ("far", far)):
                o = torch.full((bs.n_entries,), float("nan"), dtype=dt, device="cuda")
                outs[(kernel, nm)] = o
                jobs[nm].append(block_job(pkg, mid, bs, kernel, kappa, ql, o))
        # a fixed-order job beside the learned ones
        fixed = torch.full((near.n_entries,), float("nan"), dtype=torch.float64, device="cuda")
        outs["fixed"] = fixed
        counts = np.zeros(6, np.int64)
        if how == "calls":
            for nm in ("near", "far"):
                for j in jobs[nm]:
                    (ctx.bem_near_field if nm == "near" else ctx.bem_coupling_blocks)([j])
                    counts += ctx.bem_learned_counts()
            ctx.bem_near_field([block_job(pkg, mid, near, "laplace_slp", 0.0, qf, fixed)])
        else:
            plan = ctx.bem_plan_create(jobs["near"] + [block_job(pkg, mid, near, "laplace_slp",
                                                                 0.0, qf, fixed)],
                                       jobs["far"], pkg.PLAN_GRAPH)
            ctx.bem_plan_run(plan)
            counts += np.array(ctx.bem_plan_learned_counts(plan))
            ctx.bem_plan_destroy(plan)
        ctx.bem_sync()
        res[how] = ({k: v.cpu() for k, v in outs.items()}, counts)
    for k in res["calls"][0]:
        assert torch.isfinite(res["plan"][0][k]).all()
        assert torch.equal(res["calls"][0][k], res["plan"][0][k]), k
    assert np.array_equal(res["calls"][1], res["plan"][1]) and res["plan"][1].sum() > 0
    ctx.bem_set_order_model(None, 0.0)
    ctx.bem_mesh_free(mid)


def test_labels_and_normalisation_in_the_library(env):
    """bem_order_labels against the oracle's own class errors (the same rules,
    the same reference order and scale), and bem_mlp_fit_norm against the
    features' mean and standard deviation."""
    import torch
    import oracle
    pkg, ctx, om = env
    mesh = synth.jitter(synth.octasphere(12), 0.05, 151007244 + 5097)
    _, near, far = synth.workloads.h2_blocks(mesh, "p0", 32, 2.0, 16, 7)
    rng = synth.SplitMix64(11)
    a, b = _regular_pairs(mesh, (near, far), 400, rng)
    mid = ctx.bem_mesh_upload(mesh.verts, mesh.tris, "p0")
    ad, bd = to_dev(a, torch.int32), to_dev(b, torch.int32)
    classes = [("duffy", 2), ("tri7", 3), ("duffy", 4), ("duffy", 5), ("duffy", 6), ("duffy", 8)]
    for kernel, kappa in KERNELS:
        lab, err = om.labels(ctx, mid, pkg.kernel_desc(kernel, kappa), ad, bd, tol=1e-7)
        got_err = err.cpu().numpy()
        q12 = dict(q_regular=12, regular_rule="duffy", q_identical=5, q_edge=5, q_vertex=5)
        ref = oracle.entries(mesh.verts, mesh.tris, a, b, kernel=kernel, kappa=kappa, **q12)
        A = oracle.entries_absolute(mesh.verts, mesh.tris, a, b, kernel=kernel, kappa=kappa, **q12)
        E = np.stack([np.abs(oracle.entries(mesh.verts, mesh.tris, a, b, kernel=kernel,
                                            kappa=kappa, **dict(q12, regular_rule=r, q_regular=q))
                             - ref) / A for r, q in classes], axis=1)
        assert np.allclose(got_err, E, rtol=1e-4, atol=1e-12)
        ok = E <= 1e-7
        exp = np.where(ok.any(axis=1), np.argmax(ok, axis=1), 5)
        clear = np.all(np.abs(E / 1e-7 - 1.0) > 1e-3, axis=1)   # no error at the threshold
        assert np.array_equal(lab.cpu().numpy()[clear], exp[clear])
        X = om.raw_features(ctx, mid, pkg.kernel_desc(kernel, kappa), ad, bd)
        mlp = ctx.bem_mlp_create(1)
        ctx.bem_mlp_fit_norm(mlp, X)
        _, norm = ctx.bem_mlp_get_params(mlp)
        Xh = X.cpu().numpy().astype(np.float64)
        sd = Xh.std(axis=0)
        assert np.allclose(norm[:8], Xh.mean(axis=0), rtol=1e-5, atol=1e-6)
        assert np.allclose(norm[8:], np.where(sd > 1e-6, 1.0 / np.where(sd > 0, sd, 1), 1.0),
                           rtol=1e-5)
        ctx.bem_mlp_destroy(mlp)
    ctx.bem_mesh_free(mid)
