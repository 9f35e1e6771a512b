"""GPU factorized render (Eq. 5, 8), tone-mapped loss (Eq. 14), backward
kernel and autograd wrapper vs the FP64 oracle; per-triangle error
(Sec. 4.4) vs the oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from workloads import material_params, shading_tables

pytestmark = pytest.mark.gpu

GRID = [0.02, 0.1, 0.25, 0.5, 0.75, 1.0]
REL = 1e-4


@pytest.fixture(scope="module")
def fipt():
    import paper_2304_05669_gb300 as F
    return F


def close(g, o, rel=REL):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    scale = np.maximum(np.abs(o), np.mean(np.abs(o)))
    err = np.abs(g - o) / scale
    assert err.max() <= rel, (err.max(), np.unravel_index(err.argmax(), err.shape))
    return float(err.max())


def inputs(N, seed):
    Ld, Ls0, Ls1 = shading_tables(N, len(GRID), seed=seed)
    mp = material_params(N, seed=seed + 1)
    gt = material_params(N, seed=seed + 2)
    Lgt, _ = O.render_forward(Ld, Ls0, Ls1, GRID, gt["albedo"], gt["rough"], gt["metal"])
    mask = (np.random.default_rng(seed).random(N) < 0.9).astype(np.uint8)
    return Ld, Ls0, Ls1, mp, Lgt.astype(np.float32), mask


def cu(*a):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a]


@pytest.mark.parametrize("N", [1, 1000, 65537])
def test_render_forward_and_loss(fipt, N):
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 10)
    Lr_o, loss_o = O.render_forward(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"],
                                    Lgt, mask)
    t = cu(Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask)
    Lr, loss = fipt.render_fwd(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6], t[7])
    close(Lr.cpu().numpy(), Lr_o)
    assert abs(loss.item() - loss_o) <= REL * abs(loss_o)


def test_render_full_size(fipt):
    """Forward, loss and backward over all 6,389,760 pixels of the
    differentiation configuration (24 views at 640x416), element by element."""
    N = 24 * 640 * 416
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 30)
    t = cu(Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt)
    Lr, loss = fipt.render_fwd(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6])
    ga, gs, gm = fipt.render_bwd(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6])
    Lr_o, loss_o = O.render_forward(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"], Lgt)
    close(Lr.cpu().numpy(), Lr_o)
    assert abs(loss.item() - loss_o) <= REL * abs(loss_o)
    del Lr_o
    for got, ref in zip((ga, gs, gm), O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"],
                                                     mp["metal"], Lgt)):
        close(got.cpu().numpy(), ref)


def test_render_backward_matches_analytic_gradient(fipt):
    N = 200003
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 20)
    ga_o, gs_o, gm_o = O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"],
                                     Lgt, mask, grad_scale=0.5)
    t = cu(Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask)
    scale = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    ga, gs, gm = fipt.render_bwd(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6], t[7], scale)
    close(ga.cpu().numpy(), ga_o)
    close(gs.cpu().numpy(), gs_o)
    close(gm.cpu().numpy(), gm_o)


def test_autograd_function_and_finite_differences(fipt):
    """The torch.autograd.Function's gradient on 1024 sampled points vs
    central differences of the oracle's FP64 loss."""
    N = 50000
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 30)
    t = cu(Ld, Ls0, Ls1, Lgt, mask)
    a = torch.from_numpy(mp["albedo"]).cuda().requires_grad_()
    r = torch.from_numpy(mp["rough"]).cuda().requires_grad_()
    m = torch.from_numpy(mp["metal"]).cuda().requires_grad_()
    loss = fipt.factorized_render_loss(a, r, m, (t[0], t[1], t[2]), t[3], GRID, mask=t[4])
    (2.0 * loss).backward()
    rng = np.random.default_rng(3)
    idx = rng.choice(N, 1024, replace=False)
    h = 1e-6
    G = np.array(GRID)
    keep = (np.min(np.abs(mp["rough"][idx, None] - G[None]), axis=1) > 4 * h)

    def point_loss(al, ro, me, sel):
        Lr, _ = O.render_forward(Ld[sel], Ls0[sel], Ls1[sel], GRID, al, ro, me)
        d = (O.tonemap(Lr) - O.tonemap(Lgt[sel])) ** 2
        return d.sum(1) * mask[sel]

    al = mp["albedo"][idx].astype(np.float64)
    ro = mp["rough"][idx].astype(np.float64)
    me = mp["metal"][idx].astype(np.float64)
    fd_r = 2 * (point_loss(al, ro + h, me, idx) - point_loss(al, ro - h, me, idx)) / (2 * h)
    fd_m = 2 * (point_loss(al, ro, me + h, idx) - point_loss(al, ro, me - h, idx)) / (2 * h)
    e = np.zeros_like(al)
    e[:, 1] = h
    fd_a = 2 * (point_loss(al + e, ro, me, idx) - point_loss(al - e, ro, me, idx)) / (2 * h)
    close(r.grad.cpu().numpy()[idx][keep], fd_r[keep], rel=1e-3)
    close(m.grad.cpu().numpy()[idx], fd_m, rel=1e-3)
    close(a.grad.cpu().numpy()[idx, 1], fd_a, rel=1e-3)
    ga_o, gs_o, gm_o = O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"],
                                     Lgt, mask, grad_scale=2.0)
    close(a.grad.cpu().numpy(), ga_o)
    close(r.grad.cpu().numpy(), gs_o)
    close(m.grad.cpu().numpy(), gm_o)


@pytest.mark.parametrize("P,T", [(5, 3), (100000, 36), (4194304, 2045464)])
def test_tri_error_matches_oracle(fipt, P, T):
    rng = np.random.default_rng(P)
    tri = rng.integers(-1, T, P).astype(np.int32)
    Lr = rng.random((P, 3)).astype(np.float32) * 5
    Lgt = rng.random((P, 3)).astype(np.float32) * 5
    err, cnt = fipt.tri_error(*cu(tri, Lr, Lgt), T)
    e_o, c_o = O.tri_error(tri, Lr, Lgt, T)
    assert np.array_equal(cnt.cpu().numpy(), c_o)
    assert np.allclose(err.cpu().numpy(), e_o, rtol=1e-12, atol=0)
    err2, _ = fipt.tri_error(*cu(tri, Lr, Lgt), T)
    assert torch.equal(err, err2)        # deterministic


@pytest.mark.parametrize("grid", [[0.1, 0.9], [0.02, 0.05, 0.1, 0.2, 0.35, 0.5, 0.75, 1.0]])
def test_render_grid_sizes(fipt, grid):
    """The smallest (K = 2) and the largest (K = 8) roughness grids, forward,
    loss and backward; K = 1 and K = 9 are rejected."""
    N = 4099
    Ld, Ls0, Ls1 = shading_tables(N, len(grid), seed=40)
    mp = material_params(N, seed=41)
    gt = material_params(N, seed=42)
    Lgt, _ = O.render_forward(Ld, Ls0, Ls1, grid, gt["albedo"], gt["rough"], gt["metal"])
    Lgt = Lgt.astype(np.float32)
    t = cu(Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt)
    Lr, loss = fipt.render_fwd(t[0], t[1], t[2], grid, t[3], t[4], t[5], t[6])
    Lr_o, loss_o = O.render_forward(Ld, Ls0, Ls1, grid, mp["albedo"], mp["rough"], mp["metal"], Lgt)
    close(Lr.cpu().numpy(), Lr_o)
    assert abs(loss.item() - loss_o) <= REL * abs(loss_o)
    for got, ref in zip(fipt.render_bwd(t[0], t[1], t[2], grid, t[3], t[4], t[5], t[6]),
                        O.render_grad(Ld, Ls0, Ls1, grid, mp["albedo"], mp["rough"], mp["metal"], Lgt)):
        close(got.cpu().numpy(), ref)
    with pytest.raises(fipt.FiptError):
        fipt.render_fwd(t[0], t[1][:, :1].contiguous(), t[2][:, :1].contiguous(), [0.5], t[3], t[4], t[5])


@pytest.mark.parametrize("N,with_mask", [(1, False), (65537, True), (200003, False)])
def test_fused_forward_gradient(fipt, N, with_mask):
    """render_fwd_grad (one pass) gives render_fwd's Lr and loss and
    render_bwd's gradients for an upstream gradient of 1, and the oracle's;
    render_grad_scale by 1 leaves them untouched, by 0.5 gives the oracle's
    gradients at grad_scale 0.5."""
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 50)
    mk = mask if with_mask else None
    t = cu(Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask)
    m_t = t[7] if with_mask else None
    Lr, loss, grads = fipt.render_fwd_grad(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6], m_t)
    Lr1, loss1 = fipt.render_fwd(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6], m_t)
    close(Lr.cpu().numpy(), Lr1.cpu().numpy(), rel=1e-6)
    assert abs(loss.item() - loss1.item()) <= 1e-6 * abs(loss1.item())
    for x, y in zip(grads, fipt.render_bwd(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6], m_t)):
        close(x.cpu().numpy(), y.cpu().numpy(), rel=1e-6)
    Lr_o, loss_o = O.render_forward(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"], Lgt, mk)
    close(Lr.cpu().numpy(), Lr_o)
    assert abs(loss.item() - loss_o) <= REL * abs(loss_o)
    for got, ref in zip(grads, O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"],
                                             Lgt, mk)):
        close(got.cpu().numpy(), ref)
    before = [x.clone() for x in grads]
    fipt.render_grad_scale(grads, torch.ones(1, dtype=torch.float64, device="cuda"))
    assert all(torch.equal(x, y) for x, y in zip(grads, before))
    fipt.render_grad_scale(grads, torch.full((1,), 0.5, dtype=torch.float64, device="cuda"))
    for got, ref in zip(grads, O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"],
                                             Lgt, mk, grad_scale=0.5)):
        close(got.cpu().numpy(), ref)


def test_autograd_backward_twice_and_without_grad(fipt):
    """The autograd function hands out the forward pass's gradient once; a
    second backward through the same graph recomputes it, so two leave
    twice the gradient.  Under no_grad the loss is the same."""
    N = 4099
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 60)
    t = cu(Ld, Ls0, Ls1, Lgt)
    a = torch.from_numpy(mp["albedo"]).cuda().requires_grad_()
    r = torch.from_numpy(mp["rough"]).cuda().requires_grad_()
    m = torch.from_numpy(mp["metal"]).cuda().requires_grad_()
    loss = fipt.factorized_render_loss(a, r, m, (t[0], t[1], t[2]), t[3], GRID)
    loss.backward(retain_graph=True)
    loss.backward()
    for got, ref in zip((a.grad, r.grad, m.grad),
                        O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"], Lgt,
                                      grad_scale=2.0)):
        close(got.cpu().numpy(), ref)
    with torch.no_grad():
        l2 = fipt.factorized_render_loss(a, r, m, (t[0], t[1], t[2]), t[3], GRID)
    assert abs(l2.item() - loss.item()) <= 1e-6 * abs(loss.item())


def test_render_fwd_grad_full_size(fipt):
    """The training step's fused pass (forward, loss and gradient in one
    kernel) and its upstream-gradient scale over all 6,389,760 pixels of the
    differentiation configuration, element by element against the oracle,
    with the emitter mask, and then scaled by an upstream gradient of 0.75."""
    N = 24 * 640 * 416
    Ld, Ls0, Ls1, mp, Lgt, mask = inputs(N, 31)
    t = cu(Ld, Ls0, Ls1, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask)
    Lr, loss, grads = fipt.render_fwd_grad(t[0], t[1], t[2], GRID, t[3], t[4], t[5], t[6], t[7])
    fipt.context().sync_status()
    Lr_o, loss_o = O.render_forward(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask)
    close(Lr.cpu().numpy(), Lr_o)
    assert abs(loss.item() - loss_o) <= REL * abs(loss_o)
    del Lr_o, Lr
    refs = O.render_grad(Ld, Ls0, Ls1, GRID, mp["albedo"], mp["rough"], mp["metal"], Lgt, mask)
    for got, ref in zip(grads, refs):
        close(got.cpu().numpy(), ref)
    fipt.render_grad_scale(grads, torch.full((1,), 0.75, dtype=torch.float64, device="cuda"))
    for got, ref in zip(grads, refs):
        close(got.cpu().numpy(), 0.75 * ref)
