"""The learned activation proposer: the network kernels against the FP64
network reference (forward, BF16 forward, loss and gradient, training), the
frontier features against the FP64 oracle's state, and the proposer in the
step (bit-identical results, prepared blocks used)."""
import numpy as np
import pytest

from gpu_helpers import oracle_of
from oracle import mlp_oracle as M
from paper_1510_03560_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    from paper_1510_03560_gb300 import build as B
    B.build()
    from paper_1510_03560_gb300 import lbm
    assert torch.cuda.is_available()
    return lbm


def _net(seed=7, n=300):
    rng = np.random.default_rng(seed)
    params = M.init_params(seed)
    params[M.NI * M.NH:M.NI * M.NH + M.NH] = rng.normal(0, 0.1, M.NH)
    x = rng.normal(0.0, 1.0, (n, M.NI)).astype(np.float32)
    x[:, 8:] = (rng.random((n, 26)) < 0.5)  # flag-like inputs
    y = (rng.random(n) < 0.3).astype(np.float32)
    mean = rng.normal(0.0, 0.1, M.NI).astype(np.float32)
    scale = rng.uniform(0.5, 2.0, M.NI).astype(np.float32)
    return params.astype(np.float32), x, y, mean, scale


def _mlp(L, params, mean, scale, n):
    m = L.MLP(n)
    m.set_params(params)
    m.set_scaling(mean, scale)
    return m


def test_forward_matches_reference(L):
    import torch
    params, x, y, mean, scale = _net()
    m = _mlp(L, params, mean, scale, len(y))
    got = m.forward(torch.tensor(x, device="cuda")).cpu().numpy()
    want, _ = M.forward(params.astype(np.float64), x.astype(np.float64), mean, scale)
    np.testing.assert_allclose(got, want, rtol=0, atol=2e-6)
    m.close()


def test_bf16_forward_error_bound(L):
    """bfloat16 operands (8-bit significand, relative rounding 2^-9) with
    FP32 accumulation: the probabilities stay within 0.02 of FP64."""
    import torch
    params, x, y, mean, scale = _net(seed=8)
    m = _mlp(L, params, mean, scale, len(y))
    got = m.forward(torch.tensor(x, device="cuda"), bf16=True).cpu().numpy()
    want, _ = M.forward(params.astype(np.float64), x.astype(np.float64), mean, scale)
    err = np.abs(got - want).max()
    print(f"bf16 forward: max |p - p_fp64| = {err:.3g}")
    assert err <= 0.02
    m.close()


def test_loss_and_gradient_match_reference(L):
    import torch
    params, x, y, mean, scale = _net(seed=9)
    m = _mlp(L, params, mean, scale, len(y))
    loss, g = m.loss_grad(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"),
                          want_grad=True)
    p64, x64 = params.astype(np.float64), x.astype(np.float64)
    want_loss = M.loss(p64, x64, y, mean, scale)
    want = M.grad(p64, x64, y, mean, scale)
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    err = np.abs(g - want).max()
    print(f"gradient: max |g - g_fp64| = {err:.3g} (max |g| = {np.abs(want).max():.3g})")
    assert err <= 1e-4 * np.abs(want).max() + 1e-7
    m.close()


def test_training_learns_and_is_reproducible(L):
    """A separable problem (label = first input > 0): Adam on the library's
    kernels brings the loss down, and two runs give the same parameters."""
    import torch
    rng = np.random.default_rng(11)
    x = rng.normal(0.0, 1.0, (2048, M.NI)).astype(np.float32)
    y = (x[:, 0] > 0).astype(np.float32)
    xt, yt = torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda")
    runs = []
    for _ in range(2):
        m = _mlp(L, M.init_params(2).astype(np.float32), np.zeros(M.NI, np.float32),
                 np.ones(M.NI, np.float32), 512)
        first = None
        for t in range(1, 201):
            b = slice(((t - 1) % 4) * 512, ((t - 1) % 4 + 1) * 512)
            loss, _ = m.loss_grad(xt[b], yt[b])
            first = loss if first is None else first
            m.adam(3e-3, t)
        final, _ = m.loss_grad(xt[:512], yt[:512])
        runs.append((first, final, m.params()))
        m.close()
    print(f"training: loss {runs[0][0]:.4f} -> {runs[0][1]:.4f}")
    assert runs[0][1] < 0.1 < runs[0][0]
    np.testing.assert_array_equal(runs[0][2], runs[1][2])


def oracle_features(orc, case, ids):
    """The 34 features of include/lbm.h from the oracle's state: moments of
    the next streaming (rho, and j = rho u_phys - F / 2), meshed flags."""
    ct = case["cell_type"]
    nz, ny, nx = ct.shape
    nb = (nx // 8, ny // 8, nz // 8)
    per = case["params"].get("periodic", (1, 1, 0))
    act = set(orc.active_blocks().tolist())
    mac = [orc.macro(a) for a in range(2)]
    F = [orc.forces(a) for a in range(2)]

    def nbr(b, d):
        q = [b % nb[0], (b // nb[0]) % nb[1], b // (nb[0] * nb[1])]
        for a in range(3):
            q[a] += d[a]
            if q[a] < 0 or q[a] >= nb[a]:
                if not per[a]:
                    return None
                q[a] %= nb[a]
        return q[0] + nb[0] * (q[1] + nb[1] * q[2])

    out = np.zeros((len(ids), 34))
    for r, b in enumerate(ids):
        f = out[r]
        i = 8
        for k in range(27):
            if k == 13:
                continue
            d = (k % 3 - 1, (k // 3) % 3 - 1, k // 9 - 1)
            nid = nbr(b, d)
            f[i] = 1.0 if (nid is not None and nid in act) else 0.0
            i += 1
        s0 = s1 = cnt = 0.0
        for w in range(6):
            axis, sgn = w >> 1, (1 if w & 1 else -1)
            d = [0, 0, 0]
            d[axis] = sgn
            nid = nbr(b, d)
            flux = 0.0
            if nid is not None and nid in act:
                q = (nid % nb[0], (nid // nb[0]) % nb[1], nid // (nb[0] * nb[1]))
                layer = 7 if sgn < 0 else 0
                for v in range(8):
                    for u in range(8):
                        loc = [u, v, 0] if axis == 2 else ([u, 0, v] if axis == 1 else [0, u, v])
                        loc[axis] = layer
                        x, y, z = (q[0] * 8 + loc[0], q[1] * 8 + loc[1], q[2] * 8 + loc[2])
                        if ct[z, y, x] != 0:
                            continue
                        s0 += mac[0][0][z, y, x]
                        s1 += mac[1][0][z, y, x]
                        cnt += 1
                        j = 0.0
                        for a in range(2):
                            j += mac[a][0][z, y, x] * mac[a][1 + axis][z, y, x] - 0.5 * F[a][z, y, x, axis]
                        flux -= sgn * j
            f[2 + w] = flux
        f[0] = s0 / cnt if cnt else case["rho_amb"][0]
        f[1] = s1 / cnt if cnt else case["rho_amb"][1]
    return out


@pytest.mark.parametrize("which", ["drop", "porous"])
def test_frontier_features_match_oracle(L, which):
    if which == "drop":
        case, steps = W.drop_in_box(), 5
    else:
        case, steps = W.porous_injection(n=(56, 40, 48), seed=1510035603, inlet=16, x_free=6,
                                         r_range=(3.0, 6.0), S=1e-4), 30
    gpu = L.from_case(case)
    orc = oracle_of(case)
    gpu.step(steps)
    orc.step(steps)
    np.testing.assert_array_equal(gpu.active_blocks(), orc.active_blocks())
    ids, feat = gpu.frontier_features()
    assert len(ids) > 0
    want = oracle_features(orc, case, ids)
    np.testing.assert_array_equal(feat[:, 8:], want[:, 8:])
    np.testing.assert_allclose(feat[:, :2], want[:, :2], rtol=1e-4)
    scale = max(1.0, np.abs(want[:, 2:8]).max())
    np.testing.assert_allclose(feat[:, 2:8], want[:, 2:8], rtol=0, atol=1e-4 * scale)
    print(f"features {which}: {len(ids)} frontier blocks, max |flux| {np.abs(want[:, 2:8]).max():.3g}")
    # every frontier block is unmeshed and borders a meshed block
    act = set(gpu.active_blocks().tolist())
    assert not (set(ids.tolist()) & act)
    gpu.close()


def test_activation_steps_match_the_mesh(L):
    case = W.drop_in_box()
    gpu = L.from_case(case)
    a0 = gpu.activation_steps()
    np.testing.assert_array_equal(np.nonzero(a0 == 0)[0], gpu.active_blocks())
    gpu.step(60)
    a = gpu.activation_steps()
    np.testing.assert_array_equal(np.nonzero(a >= 0)[0], gpu.active_blocks())
    assert a.max() <= 60
    st = gpu.stats()
    assert st["created_blocks"] == int(np.sum(a > 0))
    gpu.close()


@pytest.mark.parametrize("storage", ["fp32", "fp16"])
def test_proposer_results_are_bit_identical(L, storage):
    """Prepared solid words equal the ones computed at creation: with the
    proposer (every frontier block prepared, threshold -1) the fields and
    meshed sets are bitwise those of the run without it."""
    case = W.porous_injection(n=(64, 64, 64), seed=1510035603, inlet=16, x_free=16)
    base = L.from_case(case, storage=storage)
    prop = L.from_case(case, storage=storage)
    params, _, _, mean, scale = _net(seed=3)
    m = _mlp(L, params, mean, scale, 1)
    prop.set_proposer(m, period=4, threshold=-1.0)
    for _ in range(6):
        base.step(20)
        prop.step(20)
        np.testing.assert_array_equal(base.active_blocks(), prop.active_blocks())
    for a in range(2):
        for x, y in zip(base.macro(a), prop.macro(a)):
            np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(base.mass(), prop.mass())
    st = prop.stats()
    print(f"proposer {storage}: created {st['created_blocks']}, prepared {st['prepared_blocks']}, "
          f"hits {st['prepared_hits']}")
    assert st["created_blocks"] > 0
    assert 0 < st["prepared_hits"] <= st["created_blocks"]
    assert base.stats()["prepared_hits"] == 0
    prop.set_proposer(None)
    prop.close()
    base.close()
    m.close()


def test_trained_proposer_gain(L):
    """What the trained network buys: the 256^3 injection recipe at 128^3
    with a sphere seed it was not trained on, through the growth of the
    mesh, with and without the proposer (period 16, threshold 0.5).  The
    results are bit-identical; the test reports the block-creation time with
    and without, the share of created blocks that had been prepared, and the
    bound on any gain, 1 / (1 - creation share of the step time): the
    proposer can only take work out of block creation."""
    from paper_1510_03560_gb300 import proposer as PR
    case = PR.trace_case(1510035620, 128)
    runs = {}
    for name in ("without", "with"):
        sim = L.from_case(case)
        mlp = PR.load_model(L) if name == "with" else None
        if mlp is not None:
            sim.set_proposer(mlp, period=16, threshold=0.5)
        sim.set_profiling(True)
        sim.step(400)
        st = sim.stats()
        runs[name] = dict(stats=st, act=sim.active_blocks(), rho=[sim.macro(a)[0] for a in range(2)],
                          mass=sim.mass())
        sim.set_proposer(None)
        sim.close()
        if mlp is not None:
            mlp.close()
    a, b = runs["without"], runs["with"]
    np.testing.assert_array_equal(a["act"], b["act"])
    for x, y in zip(a["rho"], b["rho"]):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a["mass"], b["mass"])
    sa, sb = a["stats"], b["stats"]
    share = sa["kernel_ms"][1] / sum(sa["kernel_ms"])
    bound = 1.0 / (1.0 - share)
    hit = sb["prepared_hits"] / max(sb["created_blocks"], 1)
    precision = sb["prepared_hits"] / max(sb["prepared_blocks"], 1)
    print(f"trained proposer, 128^3, 400 steps: created {sb['created_blocks']}, prepared "
          f"{sb['prepared_blocks']}, hits {sb['prepared_hits']} ({hit:.0%} of created, {precision:.0%} of "
          f"prepared); creation {sa['kernel_ms'][1]:.2f} ms without, {sb['kernel_ms'][1]:.2f} ms with; "
          f"creation share {share:.1%}, so no proposer of this kind can exceed {bound:.3f}x")
    assert sb["created_blocks"] == sa["created_blocks"] > 0
    assert sb["prepared_hits"] > 0
    assert hit > 0.2 and precision > 0.3
