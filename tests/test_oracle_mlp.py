"""Pins of the FP64 MLP oracle (the learned inverse-map proposal) to what fixes it independently:
library routines for GELU and bfloat16 rounding, closed forms of degenerate networks, the
permutation symmetry of hidden units, finite differences for the hand-written backward pass, the
closed form of Adam's first steps, and the ray geometry for the entry-point coordinates."""
import math

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")


def rand_theta(seed, scale=0.3):
    g = np.random.default_rng(seed)
    th = g.standard_normal(O.MLP_NPARAM) * scale
    return th


def offsets():
    H, I, OUT = O.MLP_H, O.MLP_IN, O.MLP_OUT
    w1 = 0
    b1 = w1 + H * I
    w2 = b1 + H
    b2 = w2 + H * H
    w3 = b2 + H
    b3 = w3 + H * H
    w4 = b3 + H
    b4 = w4 + OUT * H
    return dict(w1=w1, b1=b1, w2=w2, b2=b2, w3=w3, b3=b3, w4=w4, b4=b4)


def test_gelu_matches_library_tanh_form():
    z = torch.linspace(-8, 8, 801, dtype=torch.float64, requires_grad=True)
    ref = torch.nn.functional.gelu(z, approximate="tanh")
    (gref,) = torch.autograd.grad(ref.sum(), z)
    got = np.array([O.gelu(v) for v in z.detach().numpy()])
    gg = np.array([O.gelu_grad(v) for v in z.detach().numpy()])
    assert np.abs(got - ref.detach().numpy()).max() < 1e-15
    assert np.abs(gg - gref.numpy()).max() < 1e-14
    assert O.gelu(0.0) == 0.0 and O.gelu_grad(0.0) == 0.5


def test_bf16_rounding_matches_library():
    g = np.random.default_rng(3)
    v = np.concatenate([g.standard_normal(2000) * 10 ** g.uniform(-6, 6, 2000),
                        [1.0 + 2 ** -9, 1.0 + 3 * 2 ** -9, -0.0, 65504.0, 1e-40]])
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([O.round_bf16(x) for x in v])
    assert np.array_equal(got, ref)


def test_forward_degenerate_networks_closed_form():
    off = offsets()
    th = rand_theta(1)
    x = np.random.default_rng(2).standard_normal((5, O.MLP_IN))
    # zero last layer: the output is its bias
    t0 = th.copy()
    t0[off["w4"]:off["b4"]] = 0.0
    y = O.mlp_forward(t0, x)
    assert np.array_equal(y, np.tile(t0[off["b4"]:], (5, 1)))
    # zero middle layers: y = W4 g(b3) + b4 for every input
    t1 = th.copy()
    t1[off["w3"]:off["b3"]] = 0.0
    y = O.mlp_forward(t1, x)
    h3 = np.array([O.gelu(b) for b in t1[off["b3"]:off["w4"]]])
    W4 = t1[off["w4"]:off["b4"]].reshape(O.MLP_OUT, O.MLP_H)
    ref = W4 @ h3 + t1[off["b4"]:]
    assert np.allclose(y, np.tile(ref, (5, 1)), rtol=1e-13, atol=1e-13)


def test_forward_hidden_permutation_invariance():
    """Relabelling the hidden units of layer 1 (rows of W1, b1 and columns of W2) and of layer 2
    (rows of W2, b2, columns of W3) leaves the network's function unchanged; a transposed weight
    access would not."""
    off = offsets()
    H, I = O.MLP_H, O.MLP_IN
    th = rand_theta(4)
    x = np.random.default_rng(5).standard_normal((7, I))
    y = O.mlp_forward(th, x)
    g = np.random.default_rng(6)
    p1, p2 = g.permutation(H), g.permutation(H)
    t = th.copy()
    W1 = th[off["w1"]:off["b1"]].reshape(H, I)
    W2 = th[off["w2"]:off["b2"]].reshape(H, H)
    W3 = th[off["w3"]:off["b3"]].reshape(H, H)
    t[off["w1"]:off["b1"]] = W1[p1].ravel()
    t[off["b1"]:off["w2"]] = th[off["b1"]:off["w2"]][p1]
    t[off["w2"]:off["b2"]] = W2[p2][:, p1].ravel()
    t[off["b2"]:off["w3"]] = th[off["b2"]:off["w3"]][p2]
    t[off["w3"]:off["b3"]] = W3[:, p2].ravel()
    assert np.allclose(O.mlp_forward(t, x), y, rtol=1e-12, atol=1e-12)


def test_loss_closed_form_small_case():
    """Constant network (last layer zero): heads at fixed points, known logits; the loss is the
    squared distance of the labelled head plus beta times that head's cross-entropy."""
    off = offsets()
    th = rand_theta(7)
    th[off["w4"]:off["b4"]] = 0.0
    b4 = np.zeros(O.MLP_OUT)
    heads = np.array([[0.0, 0.0], [0.5, 0.5], [-0.5, 0.2], [0.9, -0.9]])
    b4[:8] = heads.ravel()
    b4[8:12] = [0.1, -0.3, 0.7, 0.0]
    th[off["b4"]:] = b4
    x = np.zeros((3, O.MLP_IN))
    target = np.array([[0.45, 0.52], [-0.4, 0.25], [2.0, 2.0], [0.0, 0.0]])
    label = np.array([2, 3, 0, 4], dtype=np.uint8)  # heads 1, 2, none, 3
    loss, _ = O.mlp_loss_grad(th, x[[0, 1, 2, 2]], target, label, beta=0.25)
    lse = math.log(sum(math.exp(v) for v in b4[8:12]))
    l0 = (0.05 ** 2 + 0.02 ** 2) + 0.25 * (lse - (-0.3))
    l1 = (0.1 ** 2 + 0.05 ** 2) + 0.25 * (lse - 0.7)
    l3 = (0.9 ** 2 + 0.9 ** 2) + 0.25 * (lse - 0.0)
    assert abs(loss - (l0 + l1 + l3) / 3) < 1e-14


def test_backward_matches_finite_differences():
    th = rand_theta(8, 0.4)
    g = np.random.default_rng(9)
    x = g.standard_normal((6, O.MLP_IN))
    target = g.uniform(-1, 1, (6, 2))
    valid = np.array([1, 2, 0, 3, 4, 1], dtype=np.uint8)
    loss, grad = O.mlp_loss_grad(th, x, target, valid, beta=0.3)
    idx = np.concatenate([g.choice(O.MLP_NPARAM, 60, replace=False), [0, O.MLP_NPARAM - 5, O.MLP_NPARAM - 9]])
    def cd(i, eps):
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        return (O.mlp_loss_grad(tp, x, target, valid, beta=0.3)[0] -
                O.mlp_loss_grad(tm, x, target, valid, beta=0.3)[0]) / (2 * eps)

    for i in idx:
        fd = (4 * cd(i, 2.5e-4) - cd(i, 5e-4)) / 3  # Richardson: O(eps^4)
        # roundoff of the differences: 1e-16 loss / eps
        assert abs(fd - grad[i]) <= 1e-8 * max(1.0, abs(grad[i])) + 1e-12 * loss, (i, fd, grad[i])


def test_adam_first_steps_closed_form():
    """With bias correction, a constant gradient moves every parameter by lr sign(g) per step
    (up to eps)."""
    n = 50
    g = np.random.default_rng(10).standard_normal(n)
    th = np.zeros(n)
    m, v = np.zeros(n), np.zeros(n)
    for t in (1, 2, 3):
        O.mlp_adam(th, m, v, g, t, lr=1e-2, eps=1e-12)
        assert np.allclose(th, -1e-2 * t * np.sign(g), rtol=0, atol=1e-12)


def test_entry_coordinates_unit_disk():
    """uv maps the projected section onto the unit disk: the centre to 0, the silhouette to
    |uv| = 1 (rays just inside hit the object, rays just outside miss), and back."""
    from paper_2403_13856_gb300 import workloads as W

    s = W.ELLIPSOID
    o = O.Object(s["a"], s["b"], s["c"], quat=s["quat"], m=s["m"], wavelength=s["wavelength"])
    assert np.allclose(O.xy_to_uv(o, 0.0, 0.0), 0.0)
    for ang in np.linspace(0, 2 * np.pi, 13)[:-1]:
        uv = np.array([np.cos(ang), np.sin(ang)])
        x, y = O.uv_to_xy(o, uv)
        assert np.allclose(O.xy_to_uv(o, x, y), uv, atol=1e-13)
        xi, yi = O.uv_to_xy(o, uv * (1 - 1e-6))
        xo, yo = O.uv_to_xy(o, uv * (1 + 1e-6))
        assert o.trace_ray(xi, yi, 0)[2] and not o.trace_ray(xo, yo, 0)[2]


def test_features_layout():
    from paper_2403_13856_gb300 import workloads as W

    s = W.ELLIPSOID
    o = O.Object(s["a"], s["b"], s["c"], quat=s["quat"], m=s["m"], wavelength=s["wavelength"])
    d = np.array([0.3, -0.4, np.sqrt(1 - 0.25)])
    f = O.mlp_features(o, d)[0]
    assert np.array_equal(f[:3], d)
    R = f[3:12].reshape(3, 3)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-14) and abs(np.linalg.det(R) - 1) < 1e-14
    # the rotation about x by 20 degrees
    c, sn = np.cos(np.radians(20)), np.sin(np.radians(20))
    assert np.allclose(R, [[1, 0, 0], [0, c, -sn], [0, sn, c]], atol=1e-14)
    assert np.allclose(f[12:15], [1.0, 100 / 120, 80 / 120]) and abs(f[15] - 0.333) < 1e-15
