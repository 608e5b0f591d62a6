"""Pins of the oracle's real-to-sim taxel regressor (appendix "Modeling Real Sensors"):
an independent torch float64 restatement from library layers, permutation invariance of the
attention pooling, softmax shift invariance, a one-node pad, constant features, and planted
mistakes.  CPU only."""
import os

import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle as O
from paper_2604_20295_gb300 import inputs as I


def _torch_regress(scene, disp, rp):
    """Restatement with torch library layers (linear, relu, tanh, softmax), FP64."""
    S = I.regressor_param_slices()
    W = {k: torch.tensor(np.asarray(rp[a:a + n], np.float64).reshape(s)) for k, (a, n, s) in S.items()}
    lin = lambda x, name: F.linear(x, W["W" + name], W["b" + name])
    out, attn = [], []
    offs = scene.node_offsets
    for p, t in enumerate(scene.pad_type):
        T = scene.types[t]
        x = torch.tensor(np.concatenate([T.pos, T.nrm, disp[offs[p]:offs[p + 1]]], 1), dtype=torch.float64)
        h3 = F.relu(lin(F.relu(lin(F.relu(lin(x, "R1")), "R2")), "R3"))
        f = h3 + F.relu(lin(h3, "R4"))
        a = lin(torch.tanh(lin(f, "A1")), "A2")[:, 0]
        al = torch.softmax(a, dim=0)
        g = (al[:, None] * f).sum(0)
        out.append(lin(F.relu(lin(g, "H1")), "H2").numpy())
        attn.append(al.numpy())
    return np.array(out), np.concatenate(attn)


def _scene_and_disp(seed=0):
    sc = I.hand_scene(8, seed=seed).subset([0, 3])
    th = I.make_params(seed)
    return sc, O.forward(sc, th)["disp"]


def test_matches_torch_restatement():
    sc, d = _scene_and_disp(1)
    rp = I.make_regressor_params(3).astype(np.float64)
    got = O.regress(sc, d, rp)
    ref, att = _torch_regress(sc, d, rp)
    np.testing.assert_allclose(got["taxels"], ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(got["attn"], att, rtol=1e-10, atol=1e-15)
    sums = np.add.reduceat(got["attn"], sc.node_offsets[:-1])
    np.testing.assert_allclose(sums, 1.0, rtol=1e-12)


def test_permutation_invariance():
    """Reordering a pad's nodes (geometry and displacement together) leaves its taxel
    outputs unchanged and permutes the attention weights with the nodes."""
    base = I.flat_pad(12, 12, 1.0)
    rng = np.random.default_rng(4)
    perm = rng.permutation(base.n)
    shuf = I.PadType("shuffled", base.rows, base.cols, base.pitch, 0.0, base.pos[perm].copy(),
                     base.nrm[perm].copy())
    obj = {0: (I.OBJ_SPHERE, (5.0, 0, 0), (0.3, -0.2, 3.9, 0, 0, 0, 1))}
    sa = I.custom_scene([base], [0], obj, [(0, 0, 0, 0, 0, 0, 1)], 1, 1)
    sb = I.custom_scene([shuf], [0], obj, [(0, 0, 0, 0, 0, 0, 1)], 1, 1)
    d = O.forward(sa, I.make_params(2))["disp"]
    rp = I.make_regressor_params(5)
    ra, rb = O.regress(sa, d, rp), O.regress(sb, d[perm], rp)
    np.testing.assert_allclose(rb["taxels"], ra["taxels"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(rb["attn"], ra["attn"][perm], rtol=1e-12, atol=1e-18)


def test_softmax_shift_invariance_and_one_node_pad():
    """Adding a constant to every attention score (the A2 bias) changes nothing; a pad of one
    node gives that node weight 1."""
    sc, d = _scene_and_disp(2)
    rp = I.make_regressor_params(6).astype(np.float64)
    a, b = O.regress(sc, d, rp), None
    rp2 = rp.copy()
    off = I.regressor_param_slices()["bA2"][0]
    rp2[off] += 7.5
    b = O.regress(sc, d, rp2)
    np.testing.assert_allclose(b["taxels"], a["taxels"], rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(b["attn"], a["attn"], rtol=1e-12, atol=1e-18)
    one = I.PadType("one", 1, 1, 1.0, 0.0, np.zeros((1, 3), np.float32),
                    np.array([[0, 0, 1]], np.float32))
    s1 = I.custom_scene([one], [0], {}, [(0, 0, 0, 0, 0, 0, 1)], 1, 1)
    r1 = O.regress(s1, np.array([[0.1, -0.2, -0.5]]), rp)
    assert r1["attn"][0] == 1.0


def test_constant_features_make_the_pooling_irrelevant():
    """With every encoder weight zero, every node's feature is the same vector
    f = relu(b3) + relu(b4 + W4 relu(b3)), so the pooled feature is f whatever the attention
    does, and the output is the head applied to f."""
    sc, d = _scene_and_disp(3)
    rp = I.make_regressor_params(8).astype(np.float64)
    S = I.regressor_param_slices()
    for name in ("WR1", "WR2", "WR3"):
        a, n, _ = S[name]
        rp[a:a + n] = 0.0
    P = {k: rp[a:a + n].reshape(s) for k, (a, n, s) in S.items()}
    h3 = np.maximum(P["bR3"], 0)
    f = h3 + np.maximum(P["WR4"] @ h3 + P["bR4"], 0)
    y = P["WH2"] @ np.maximum(P["WH1"] @ f + P["bH1"], 0) + P["bH2"]
    got = O.regress(sc, d, rp)["taxels"]
    np.testing.assert_allclose(got, np.broadcast_to(y, got.shape), rtol=1e-12, atol=1e-14)


_MUTANTS = {
    "residual_dropped": ("f[(size_t)i * 256 + k] = h3[k] + relu(h4[k]);",
                         "f[(size_t)i * 256 + k] = relu(h4[k]);"),
    "attention_relu": ("for (int k = 0; k < 128; ++k) s1[k] = tanh(s1[k]);",
                       "for (int k = 0; k < 128; ++k) s1[k] = relu(s1[k]);"),
    "softmax_unnormalised": ("double al = a[i] / Z;", "double al = a[i];"),
    "mean_pool": ("double al = a[i] / Z;", "double al = 1.0 / n;"),
    "head_relu_dropped": ("for (int k = 0; k < 128; ++k) z[k] = relu(z[k]);",
                          "(void)0;"),
    "inputs_swapped": ("x[3 + k] = nrm[3 * i + k];\n        x[6 + k] = disp[3 * (base + i) + k];",
                       "x[6 + k] = nrm[3 * i + k];\n        x[3 + k] = disp[3 * (base + i) + k];"),
    # softmax exponent with the wrong sign (weights favour the lowest scores)
    "softmax_sign": ("a[i] = exp(a[i] - mx);", "a[i] = exp(mx - a[i]);"),
    # attention scored on the encoder output before the residual layer
    "attention_before_residual": ("reg_layer(rp, 4, f + (size_t)i * 256, s1);",
                                  "reg_layer(rp, 4, h3, s1);"),
    # every layer's weight read transposed (column-major instead of out x in row-major)
    "weights_transposed": ("acc += W[(size_t)r * in + c] * x[c];",
                           "acc += W[(size_t)c * o + r] * x[c];"),
}


def _pin_checks(lib):
    sc, d = _scene_and_disp(1)
    rp = I.make_regressor_params(3).astype(np.float64)
    got = O.regress(sc, d, rp, lib=lib)
    ref, att = _torch_regress(sc, d, rp)
    yield bool(np.allclose(got["taxels"], ref, rtol=1e-10, atol=1e-12))
    yield bool(np.allclose(np.add.reduceat(got["attn"], sc.node_offsets[:-1]), 1.0, rtol=1e-12))


def test_pin_checks_pass_on_the_oracle():
    assert all(_pin_checks(None))


@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_planted_regressor_mistake_is_caught(name, tmp_path):
    src = open(os.path.join(os.path.dirname(O.__file__), "etac_oracle.c")).read()
    old, new = _MUTANTS[name]
    assert src.count(old) == 1, name
    p = tmp_path / "mut.c"
    p.write_text(src.replace(old, new))
    lib = O.load_variant(str(p), str(tmp_path / "libmut.so"))
    assert not all(_pin_checks(lib)), f"planted mistake {name} passed every regressor pin"
