"""Differentiable SP2 network (Eq. 16 in matrix form) on the GPU against the
FP64 oracle: forward layers and checkpoints, and the hand-written adjoint
(coefficient gradients and dL/dX_0)."""
import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as m

    m.init(0)
    m.set_precision("split")
    return m


def _instances(B, N, seed0):
    return [si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=seed0 + i) for i in range(B)]


def _oracle_x0(hs):
    X0 = []
    for h in hs:
        H64 = h.h32().astype(np.float64)
        lo, hi = o.gershgorin_bounds(H64)
        X0.append(o.input_layer(H64, lo, hi))
    return np.stack(X0)


def _coef(hs, L, rng, jitter):
    r = o.sp2(hs[0].h32().astype(np.float64), hs[0].n_occ, max_iter=L, refine=False)
    coef = o.sp2_branch_coefficients(r.sigmas, L)
    return coef + rng.uniform(-jitter, jitter, coef.shape)


@pytest.mark.parametrize("B,N,L,ce", [(3, 300, 6, 2), (2, 512, 9, 4)])
def test_forward_matches_oracle(sp2, B, N, L, ce):
    rng = np.random.default_rng(N)
    hs = _instances(B, N, 3000)
    coef = _coef(hs, L, rng, 0.02).astype(np.float32)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    X, ck, bounds = sp2.network_forward(H, coef, ckpt_every=ce)
    X0 = _oracle_x0(hs)
    XL, xs = o.network_forward(X0, coef.astype(np.float64), keep=True)
    err = np.max(np.abs(X.cpu().numpy() - XL))
    print(f"forward B={B} N={N} L={L}: max-abs {err:.2e}")
    assert err <= 1e-4
    for k in range(L // ce + 1):
        assert np.max(np.abs(ck[k].cpu().numpy() - xs[k * ce])) <= 1e-4
    for b, h in enumerate(hs):
        lo, hi = o.gershgorin_bounds(h.h32().astype(np.float64))
        assert abs(bounds[b, 0].item() - lo) <= 1e-6 * abs(lo) and abs(bounds[b, 1].item() - hi) <= 1e-6 * abs(hi)


@pytest.mark.parametrize("B,N,L,ce", [(2, 300, 6, 2), (2, 640, 8, 3)])
def test_adjoint_matches_oracle(sp2, B, N, L, ce):
    rng = np.random.default_rng(7 + N)
    hs = _instances(B, N, 4000)
    coef = _coef(hs, L, rng, 0.05).astype(np.float32)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    X, ck, _ = sp2.network_forward(H, coef, ckpt_every=ce)
    target = np.stack([o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 0.05) for h in hs])
    # loss = (1/B) sum_b ||X_L - D_FD||_F^2  ->  G_L = 2 (X_L - D_FD) / B
    G_L = (2.0 * (X.cpu().numpy().astype(np.float64) - target) / B).astype(np.float32)
    dcoef, G0 = sp2.network_backward(H, coef, ce, ck, torch.from_numpy(G_L).cuda())
    X0 = _oracle_x0(hs)
    want_d, want_G0 = o.network_adjoint(X0, coef.astype(np.float64), G_L.astype(np.float64))
    d = dcoef.numpy()
    rel = np.max(np.abs(d - want_d)) / np.max(np.abs(want_d))
    g0 = np.max(np.abs(G0.cpu().numpy() - want_G0)) / np.max(np.abs(want_G0))
    print(f"adjoint B={B} N={N} L={L}: dcoef rel {rel:.2e}, G0 rel {g0:.2e}")
    assert rel <= 1e-3
    assert g0 <= 1e-3


def test_autograd_function(sp2):
    rng = np.random.default_rng(1)
    hs = _instances(2, 256, 5000)
    L = 5
    coef = torch.tensor(_coef(hs, L, rng, 0.02), dtype=torch.float32, requires_grad=True)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    X = sp2.SP2Network.apply(H, coef, 1)
    target = torch.from_numpy(np.stack([o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 0.05) for h in hs])).float().cuda()
    loss = ((X - target) ** 2).sum() / 2
    loss.backward()
    X0 = _oracle_x0(hs)
    XL = o.network_forward(X0, coef.detach().numpy().astype(np.float64))
    want, _ = o.network_adjoint(X0, coef.detach().numpy().astype(np.float64), 2.0 * (XL - target.cpu().numpy()) / 2)
    assert np.max(np.abs(coef.grad.numpy() - want)) <= 1e-3 * np.max(np.abs(want))


def test_forward_ragged_size(sp2):
    """N not a multiple of 4 (scalar load/store paths of the epilogue)."""
    rng = np.random.default_rng(2)
    hs = _instances(2, 257, 3100)
    coef = _coef(hs, 5, rng, 0.02).astype(np.float32)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    X, ck, _ = sp2.network_forward(H, coef, ckpt_every=5)
    XL = o.network_forward(_oracle_x0(hs), coef.astype(np.float64))
    assert np.max(np.abs(X.cpu().numpy() - XL)) <= 1e-4


def test_training_steps_reduce_the_loss(sp2):
    """The paper's learning of layer coefficients (Sec. "Capitalizing on the
    machine learning perspective"): gradient steps through the hand-written
    adjoint lower the Frobenius loss against the Fermi-Dirac target (C14, C16)."""
    rng = np.random.default_rng(11)
    hs = _instances(3, 256, 5200)
    L = 8
    coef0 = _coef(hs, L, rng, 0.03)
    coef = torch.tensor(coef0, dtype=torch.float32, requires_grad=True)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    target = torch.from_numpy(np.stack([o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 0.05) for h in hs])).float().cuda()
    opt = torch.optim.Adam([coef], lr=2e-3)
    losses = []
    for _ in range(12):
        opt.zero_grad()
        X = sp2.SP2Network.apply(H, coef, 2)
        loss = ((X - target) ** 2).sum() / len(hs)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    print("losses:", [round(v, 4) for v in losses])
    assert losses[-1] < 0.8 * losses[0]


def test_adjoint_plain_fp16(sp2):
    """The adjoint on the plain-FP16 tensor-core path (one product per tile,
    hi planes only), segments of uneven length (L = 7, ckpt_every = 3).
    Rounding each operand to FP16 (unit roundoff 2^-11) perturbs every layer
    of forward recomputation and adjoint by about 5e-4 relative, so the
    gradients are held to 1e-2 relative instead of the split path's 1e-3."""
    rng = np.random.default_rng(13)
    hs = _instances(2, 300, 4100)
    L, ce = 7, 3
    coef = _coef(hs, L, rng, 0.05).astype(np.float32)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    sp2.set_precision("fp16")
    try:
        X, ck, _ = sp2.network_forward(H, coef, ckpt_every=ce)
        target = np.stack([o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 0.05) for h in hs])
        G_L = (2.0 * (X.cpu().numpy().astype(np.float64) - target) / len(hs)).astype(np.float32)
        dcoef, G0 = sp2.network_backward(H, coef, ce, ck, torch.from_numpy(G_L).cuda())
    finally:
        sp2.set_precision("split")
    X0 = _oracle_x0(hs)
    want_d, want_G0 = o.network_adjoint(X0, coef.astype(np.float64), G_L.astype(np.float64))
    rel = np.max(np.abs(dcoef.numpy() - want_d)) / np.max(np.abs(want_d))
    g0 = np.max(np.abs(G0.cpu().numpy() - want_G0)) / np.max(np.abs(want_G0))
    print(f"adjoint fp16: dcoef rel {rel:.2e}, G0 rel {g0:.2e}")
    assert rel <= 1e-2
    assert g0 <= 1e-2


def test_network_at_its_configuration(sp2):
    """The network workload's shape (Eq. 16 in matrix form): N = 2048, L = 20,
    checkpoints every 5 layers, coefficients at the SP2 branch values of
    instance 0's FP64 solve (C15), the Fermi-Dirac target at kT = 0.05, mu = 0
    (C14) and the squared Frobenius loss (C16); B = 4 instances keep the FP64
    oracle affordable.  Checked: X_L and every checkpoint against the oracle's
    forward; dcoef and dL/dX_0 of the hand-written adjoint against the
    oracle's FP64 adjoint; and six coefficient gradients against central
    differences (h = 1e-4) of the GPU forward with the loss summed in FP64.

    Central differences of a forward that stores X in FP32 carry an absolute
    noise floor: the two perturbed forwards round every element of every
    layer differently, which moves the loss by ~1e-6 and the quotient by a few
    1e-2 on gradients of up to ~2e2.  Their errors are therefore measured, as
    the comparison with the oracle's adjoint is, against the largest
    coefficient gradient."""
    B, N, L, ce = 4, 2048, 20, 5
    hs = [si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=2000 + i, device="cuda")
          for i in range(B)]
    r = o.sp2(hs[0].h32().astype(np.float64), hs[0].n_occ, max_iter=L, refine=False)
    coef = o.sp2_branch_coefficients(r.sigmas, L).astype(np.float32)
    H = torch.from_numpy(np.stack([h.h32() for h in hs])).cuda()
    X, ck, _ = sp2.network_forward(H, coef, ckpt_every=ce)
    X0 = _oracle_x0(hs)
    XL, xs = o.network_forward(X0, coef.astype(np.float64), keep=True)
    Xh = X.cpu().numpy().astype(np.float64)
    fwd = float(np.max(np.abs(Xh - XL)))
    ckerr = max(float(np.max(np.abs(ck[k].cpu().numpy() - xs[k * ce]))) for k in range(L // ce + 1))
    del xs
    target = np.stack([o.fermi_dirac_closed_form(h.Q, h.eps, 0.0, 0.05) for h in hs])
    G_L = (2.0 * (Xh - target) / B).astype(np.float32)
    dcoef, G0 = sp2.network_backward(H, coef, ce, ck, torch.from_numpy(G_L).cuda())
    want_d, want_G0 = o.network_adjoint(X0, coef.astype(np.float64), G_L.astype(np.float64))
    d = dcoef.numpy().astype(np.float64)
    rel_d = float(np.max(np.abs(d - want_d)) / np.max(np.abs(want_d)))
    rel_g0 = float(np.max(np.abs(G0.cpu().numpy() - want_G0)) / np.max(np.abs(want_G0)))

    T = torch.from_numpy(target).cuda()

    def loss(cf):
        Xc, _, _ = sp2.network_forward(H, cf, ckpt_every=ce)
        return float(((Xc.double() - T) ** 2).sum().item() / B)

    fd_err = 0.0
    for n, k in [(0, 0), (0, 1), (4, 2), (9, 0), (14, 1), (19, 2)]:
        cp, cm = coef.copy(), coef.copy()
        cp[n, k] = np.float32(coef[n, k] + 1e-4)
        cm[n, k] = np.float32(coef[n, k] - 1e-4)
        fd = (loss(cp) - loss(cm)) / (float(cp[n, k]) - float(cm[n, k]))
        e = abs(fd - d[n, k]) / np.max(np.abs(d))
        print(f"  coef ({n},{k}): adjoint {d[n, k]:+.6e}  central difference {fd:+.6e}  rel {e:.2e}")
        fd_err = max(fd_err, e)
    print(f"network B={B} N={N} L={L}: forward max-abs {fwd:.2e}, checkpoints {ckerr:.2e}; "
          f"adjoint vs FP64 adjoint: dcoef rel {rel_d:.2e}, G0 rel {rel_g0:.2e}; vs central differences {fd_err:.2e}")
    assert fwd <= 1e-4 and ckerr <= 1e-4
    assert rel_d <= 1e-3 and rel_g0 <= 1e-3
    assert fd_err <= 1e-3
