"""GPU parity of the (m, s)-proposing network's kernels against the numpy
oracle (forward, cross-entropy gradient, Adam), and of the learned/certified
selection path against the oracle's certified selection."""
import numpy as np
import pytest

from oracle import mlp as M

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_10989_gb300 import api as A
    return A


def _setup(api, n_in=5, hid=64, n_out=60, B=96, seed=0):
    import torch
    rng = np.random.default_rng(seed)
    net = api.MLP(n_in, hid, n_out, seed=seed)
    theta = net.params.cpu().numpy().astype(np.float64)
    theta += rng.standard_normal(theta.size) * 0.05          # non-zero biases too
    net.params.copy_(torch.from_numpy(theta.astype(np.float32)))
    theta = net.params.cpu().numpy().astype(np.float64)
    X = rng.standard_normal((B, n_in)).astype(np.float32)
    y = rng.integers(0, n_out, size=B)
    return net, theta, X, y


def test_forward_matches_oracle(api):
    import torch
    net, theta, X, _ = _setup(api)
    got = net.forward(torch.from_numpy(X).cuda()).cpu().numpy()
    want, _ = M.forward(theta, X.astype(np.float64), 5, 64, 60)
    assert np.abs(got - want).max() < 1e-5 * max(1.0, np.abs(want).max())


def test_gradient_matches_oracle(api):
    import torch
    net, theta, X, y = _setup(api, seed=1)
    g, loss = net.grad(torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda())
    wl, wg = M.loss_and_grad(theta, X.astype(np.float64), y, 5, 64, 60)
    g = g.cpu().numpy()
    assert float(loss.mean()) == pytest.approx(wl, rel=1e-5)
    assert np.linalg.norm(g - wg) / np.linalg.norm(wg) < 1e-5
    assert np.abs(g - wg).max() < 1e-4 * np.abs(wg).max()


def test_adam_step_matches_oracle(api):
    import torch
    net, theta, X, y = _setup(api, seed=2)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for step in (1, 2, 3):
        _, wg = M.loss_and_grad(theta, X.astype(np.float64), y, 5, 64, 60)
        theta, m, v = M.adam(theta, wg, m, v, step, lr=1e-3)
        net.train_step(Xd, yd, lr=1e-3)
    got = net.params.cpu().numpy()
    assert np.abs(got - theta).max() < 1e-5


def test_training_learns(api):
    import torch
    rng = np.random.default_rng(5)
    X = rng.standard_normal((2048, 5)).astype(np.float32)
    y = (np.clip(np.floor((X[:, 0] + 2.5) * 2), 0, 9)).astype(np.int64)   # 10 ordered classes
    net = api.MLP(5, 64, 10, seed=3)
    Xd, yd = torch.from_numpy(X).cuda(), torch.from_numpy(y).cuda()
    l0 = float(net.grad(Xd, yd)[1].mean())
    for _ in range(400):
        net.train_step(Xd, yd, lr=3e-3)
    l1 = float(net.grad(Xd, yd)[1].mean())
    acc = float((net.forward(Xd).argmax(1) == yd).float().mean())
    assert l1 < 0.25 * l0 and acc > 0.9


# ---- selection inside the batched launch ------------------------------------------------

def _batch(n_list, norms, seed, dtype=np.float64):
    from paper_1710_10989_gb300 import workloads as W
    return [W.batch_matrix(i, int(n), float(v), seed=seed).astype(dtype) for i, (n, v) in
            enumerate(zip(n_list, norms))]


@pytest.fixture(scope="module")
def h(api):
    hh = api.Handle(0)
    hh.batch_reserve(512)
    yield hh
    hh.close()


def test_data_mode_norms_and_features(h, api):
    import torch
    from oracle import oracle as O
    ns = [8, 33, 64, 130, 257, 300]
    mats = _batch(ns, [0.01, 3.0, 20.0, 70.0, 5.0, 0.5], seed=21)
    ins = [torch.from_numpy(A).cuda() for A in mats]
    b = api.Batch(ins)
    feat, norms = h.selector_data(b)
    feat, norms = feat.cpu().numpy(), norms.cpu().numpy()
    for A, f, nr in zip(mats, feat, norms):
        want = O.power_norms(A)
        assert np.allclose(nr[:3], want[:3], rtol=1e-13, atol=0) and np.isnan(nr[3])
        assert f[0] == pytest.approx(np.log(want[0]), abs=1e-5)
        assert f[4] == pytest.approx(np.log(A.shape[0]), abs=1e-5)
        for k in (2, 3, 4):  # random-vector estimates bound ||A^k|| from below
            assert f[k - 1] <= np.log(want[k - 1]) / k + 1e-4


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_alpha_rule_matches_oracle(h, api, dtype):
    import torch
    from oracle import oracle as O
    from paper_1710_10989_gb300 import workloads as W
    ns, nv = W.batch_spec(count=24, seed=22)
    mats = _batch(ns, nv, seed=22, dtype=dtype)
    ins = [torch.from_numpy(A).cuda() for A in mats]
    outs = [torch.zeros_like(a) for a in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b, flags=api.SELECT_ALPHA)
    torch.cuda.synchronize()
    pi = {1: 0, 2: 1, 4: 2, 8: 3, 12: 4, 18: 5}
    tol = 1e-12 if dtype == np.float64 else 1e-6
    for A, o, inf in zip(mats, outs, b.infos()):
        A = A.astype(np.float64)
        m, s = O.select_certified(O.power_norms(A))
        assert (inf["m"], inf["s"], inf["selector"]) == (m, s, 5), (inf, m, s)
        # A^2 and A^3 are computed for the bound; T12 and T18 reuse them, smaller degrees do not
        assert inf["products"] == pi[m] + s + (0 if m in (12, 18) else 2)
        E, _ = O.expm(A, m=m, s=s)
        got = o.cpu().numpy().astype(np.float64)
        assert np.linalg.norm(got - E) / np.linalg.norm(E) < tol


def test_learned_mode_is_sound_with_any_network(h, api):
    """A random (untrained) network: whatever it proposes, a choice is used only when
    certified, everything else falls back, and every result stays accurate."""
    import torch
    from oracle import oracle as O
    from paper_1710_10989_gb300 import workloads as W
    net = api.MLP(5, 64, 60, seed=11)
    h.batch_set_selector(net, 10, [0.0] * 5, [1.0] * 5)
    ns, nv = W.batch_spec(count=40, seed=23)
    mats = _batch(ns, nv, seed=23)
    ins = [torch.from_numpy(A).cuda() for A in mats]
    outs = [torch.zeros_like(a) for a in ins]
    b = api.Batch(ins, outs)
    h.expm_batched(b, flags=api.SELECT_LEARNED)
    torch.cuda.synchronize()
    th = O.theta_array("new")
    seen = set()
    for A, o, inf in zip(mats, outs, b.infos()):
        nr = O.power_norms(A)
        m, s = inf["m"], inf["s"]
        seen.add(inf["selector"])
        alpha2 = max(nr[1] ** 0.5, nr[2] ** (1 / 3))
        if inf["selector"] == 2:
            assert nr[0] / 2 ** s <= th[m]
        elif inf["selector"] == 3:
            assert alpha2 / 2 ** s <= th[m] * (1 + 1e-9)
        else:
            assert inf["selector"] == 4 and (m, s) == O.select(nr[0])
        E, _ = O.expm(A, m=m, s=s)
        got = o.cpu().numpy()
        assert np.linalg.norm(got - E) / np.linalg.norm(E) < 1e-12
    assert seen <= {2, 3, 4}


def test_trained_network_gains_over_the_plain_rule(api):
    """The committed network (trained on 10^6 generated matrices): on held-out
    matrices it needs fewer products than the paper's rule, nearly never falls
    back, and every result stays as accurate."""
    import torch
    from oracle import oracle as O
    from paper_1710_10989_gb300 import selector as SEL
    hh = api.Handle(0)
    hh.batch_reserve(512)
    SEL.install(hh)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(12)
    rng = np.random.default_rng(12)
    mats = []
    while len(mats) < 512:
        n = int(rng.integers(16, 257))
        mats += list(SEL.gpu_matrices(torch, n, 32, gen).unbind(0))
    prods, sels = {}, {}
    outs = {}
    for name, flags in (("plain", 0), ("learned", api.SELECT_LEARNED)):
        o = [torch.empty_like(a) for a in mats]
        b = api.Batch(mats, o)
        hh.expm_batched(b, flags=flags)
        torch.cuda.synchronize()
        inf = b.infos()
        prods[name] = np.mean([i["products"] for i in inf])
        sels[name] = np.array([i["selector"] for i in inf])
        outs[name] = o
    assert prods["learned"] < 0.95 * prods["plain"], prods
    assert np.mean(sels["learned"] == 4) < 0.05
    for i in range(0, 512, 64):
        A = mats[i].cpu().numpy()
        ref, _ = O.expm(A)
        for name in outs:
            got = outs[name][i].cpu().numpy()
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12
    hh.close()


def test_training_labels_relabelled_by_the_oracle(api):
    """The network's training labels come from the library's data mode (FP64
    power norms on the GPU, then bbc_select_certified). A 1 % random sample of
    10,240 matrices drawn as the training set is (N uniform on 16..512, seed 11)
    is re-labelled by the oracle (its own products for ||A^k||_1 and its own
    certified selection); the disagreement rate is reported and must stay at or
    below one sample in a hundred (a disagreement needs a norm within rounding
    of a threshold)."""
    import torch
    from oracle import oracle as O
    from paper_1710_10989_gb300 import selector as SEL
    h = api.Handle(0)
    h.batch_reserve(512)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    rng = np.random.default_rng(11)
    pick = np.random.default_rng(111)
    total, sample = 0, []
    while total < 10240:
        n = int(rng.integers(16, 513))
        A = SEL.gpu_matrices(torch, n, 256, gen)
        _, nr = h.selector_data(api.Batch(list(A.unbind(0))))
        lib_labels = SEL.labels_of(nr.cpu().numpy())
        for j in np.nonzero(pick.random(256) < 0.01)[0]:
            sample.append((A[j].cpu().numpy(), int(lib_labels[j])))
        total += 256
    h.close()
    assert len(sample) >= 80
    disagree = 0
    for Ah, lab in sample:
        m, s = O.select_certified(O.power_norms(Ah))
        disagree += lab != SEL.DEGREES.index(m) * SEL.S_VALUES + min(s, SEL.S_VALUES - 1)
    rate = disagree / len(sample)
    print(f"oracle re-label of {len(sample)} of {total} training-style matrices: disagreement rate {rate:.4f}")
    assert disagree <= max(1, len(sample) // 100), (disagree, len(sample))


def test_single_matrix_call_with_certified_selection(api):
    """bbc_expm with BBC_SELECT_LEARNED / BBC_SELECT_ALPHA (a batch of one through the
    persistent kernel): the same (m, s), products and result as the batched call, and
    the oracle's exp(A) at that (m, s); the alpha rule's (m, s) is the oracle's
    certified choice."""
    import torch
    from oracle import oracle as O
    from paper_1710_10989_gb300 import selector as SEL, workloads as W
    h = api.Handle(0)
    h.batch_reserve(512)
    SEL.install(h)
    for n, norm, seed in ((200, 3.0, 1), (64, 0.05, 2), (512, 40.0, 3)):
        A = W.batch_matrix(seed, n, norm, seed=41)
        dA = torch.from_numpy(A).cuda()
        for flag in (api.SELECT_LEARNED, api.SELECT_ALPHA):
            out = torch.empty_like(dA)
            info = h.expm(dA, out, 0.0, flag)
            ref = torch.empty_like(dA)
            b = api.Batch([dA], [ref])
            h.expm_batched(b, flags=flag)
            torch.cuda.synchronize()
            bi = b.infos()[0]
            assert (info.m, info.s, info.products, info.selector) == (bi["m"], bi["s"], bi["products"],
                                                                     bi["selector"])
            assert torch.equal(out, ref)
            want, _ = O.expm(A, m=info.m, s=info.s)
            assert np.linalg.norm(out.cpu().numpy() - want) / np.linalg.norm(want) < 1e-12
            if flag == api.SELECT_ALPHA:
                assert (info.m, info.s) == O.select_certified(O.power_norms(A))
    with pytest.raises(api.BBCError) as e:                  # beyond the reservation
        big = torch.zeros((600, 600), dtype=torch.float64, device="cuda")
        h.expm(big, torch.empty_like(big), 0.0, api.SELECT_ALPHA)
    assert e.value.code == api.INVALID_ARG
    with pytest.raises(api.BBCError) as e:                  # FP64 products only
        h.expm(dA, torch.empty_like(dA), 0.0, api.SELECT_ALPHA | api.PREC_OZAKI)
    assert e.value.code == api.UNSUPPORTED
    h.close()
