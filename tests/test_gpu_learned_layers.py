"""Learning shortens the layer count (Sec. "Capitalizing on the machine
learning perspective", point 2; Eq. 16).

A 16-layer network X_{n+1} = a_n X_n^2 + b_n X_n + c_n I, started from the
SP2 branch values of one training instance (reading C15), is trained with
Adam through the library's forward and hand-written adjoint (split-FP16
kernels) to minimise the squared Frobenius distance to the zero-temperature
density matrix (Eq. 6) of eight gapped training Hamiltonians.  On held-out
Hamiltonians from the same distribution its error is then compared with
SP2 itself, which picks every branch from the instance's own traces
(Alg. 1, the FP64 oracle): the trained 16 layers reach what SP2 needs at
least 20 layers for.  (A fixed branch sequence copied from one instance
does not carry over to another at all: its error stays near 0.1.)"""
import numpy as np
import pytest

import oracle as o
import sp2_inputs as si

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N, L = 128, 16


def _set(seed0, count):
    return [si.gapped_hamiltonian(N, N // 2, (-1.0, -0.05), (0.05, 1.0), seed=seed0 + i) for i in range(count)]


def test_trained_network_needs_fewer_layers_than_sp2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2101_06385_gb300 as sp2

    sp2.init(0)
    sp2.set_precision("split")
    train, test = _set(7000, 8), _set(8000, 4)
    Htr = torch.from_numpy(np.stack([h.h32() for h in train])).cuda()
    Hte = torch.from_numpy(np.stack([h.h32() for h in test])).cuda()
    Dtr = torch.from_numpy(np.stack([o.density_matrix_closed_form(h.Q, h.n_occ) for h in train])).float().cuda()
    Dte = np.stack([o.density_matrix_closed_form(h.Q, h.n_occ) for h in test])

    r = o.sp2(train[0].H, train[0].n_occ, max_iter=L, refine=False)
    coef = torch.tensor(o.sp2_branch_coefficients(r.sigmas, L), dtype=torch.float32, requires_grad=True)
    opt = torch.optim.Adam([coef], lr=2e-3)
    sched = torch.optim.lr_scheduler.MultiStepLR(opt, milestones=[1500, 2500], gamma=0.3)
    best, best_coef = float("inf"), None
    for _ in range(3000):
        opt.zero_grad()
        X = sp2.SP2Network.apply(Htr, coef, 4)
        loss = ((X - Dtr) ** 2).sum() / len(train)
        loss.backward()
        opt.step()
        sched.step()
        if loss.item() < best:
            best, best_coef = loss.item(), coef.detach().clone()

    with torch.no_grad():
        X, _, _ = sp2.network_forward(Hte, best_coef, 4)
    err_trained = float(np.max(np.abs(X.cpu().numpy().astype(np.float64) - Dte)))

    def sp2_err(layers):
        e = 0.0
        for h, D in zip(test, Dte):
            rr = o.sp2(h.h32().astype(np.float64), h.n_occ, max_iter=layers, refine=False)
            e = max(e, float(np.max(np.abs(rr.D - D))))
        return e

    curve = {l: sp2_err(l) for l in range(L, 33, 2)}
    match = min((l for l, e in curve.items() if e <= err_trained), default=None)
    print(f"trained {L} layers: held-out max-abs {err_trained:.2e} (training loss {best:.3e}); "
          f"SP2: " + ", ".join(f"{l}:{e:.1e}" for l, e in curve.items()) + f"; SP2 needs {match} layers for it")
    assert err_trained < curve[L]            # better than SP2 at the same depth
    assert err_trained <= curve[20]          # and at least as good as SP2 with 4 more layers
