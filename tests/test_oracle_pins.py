"""Pins for the FP64 oracle: each test checks the oracle against something other
than itself -- what the convolution's definition (paper Sec. 1 / Sec. 5.A:
six nested loops; Sec. 5.B: forward and backward passes) and plain mathematics
fix -- so that a dropped term, a wrong sign or index, or a transposed operand
fails at least one of them.

* 1x1 identity filters reproduce the input exactly;
* delta filters shift the input exactly (pins stride, padding, dilation);
* linearity in x and in w;
* integer-valued inputs give exact sums, equal to the rounded FFT result;
* brute-force FFT cross-correlation agrees to 1e-12 on tiny inputs;
* torch.nn.functional.conv2d in float64 (a library special case, test only);
* adjoint identities <conv(x,w), g> = <x, dgrad(g,w)> = <w, wgrad(x,g)>;
* central finite differences of L = sum g*y give dx, dw, db, and through
  a ReLU those of L = sum g*relu(y) (pre-activations kept off the kink);
* the quantisers against their format definitions and torch's converters.
"""
import itertools

import numpy as np
import pytest
import torch

import oracle
from oracle import Conv


def _rng(seed):
    return np.random.default_rng(seed)


def _to_layout(a_nchw, layout):
    return a_nchw if layout == "NCHW" else np.ascontiguousarray(a_nchw.transpose(0, 2, 3, 1))


def _from_layout(a, layout):
    return a if layout == "NCHW" else np.ascontiguousarray(a.transpose(0, 3, 1, 2))


def _fft_conv(x, w, b, stride, pad, dil):
    """Cross-correlation via numpy FFT on NCHW / KCRS float64 arrays.

    Correlation with w equals convolution with w flipped in both spatial axes.
    The dilated filter has d-1 zeros between taps. The stride subsamples the
    stride-1 result."""
    N, C, H, W = x.shape
    K, _, R, S = w.shape
    (u, v), (ph, pw), (dh, dw) = stride, pad, dil
    xp = np.zeros((N, C, H + 2 * ph, W + 2 * pw))
    xp[:, :, ph:ph + H, pw:pw + W] = x
    Rd, Sd = dh * (R - 1) + 1, dw * (S - 1) + 1
    wd = np.zeros((K, C, Rd, Sd))
    wd[:, :, ::dh, ::dw] = w
    Hp, Wp = xp.shape[2:]
    fh, fw = Hp + Rd - 1, Wp + Sd - 1
    X = np.fft.rfft2(xp, s=(fh, fw))                      # N C fh fw'
    Wf = np.fft.rfft2(wd[:, :, ::-1, ::-1], s=(fh, fw))   # K C fh fw'
    Y = np.einsum("ncij,kcij->nkij", X, Wf)
    full = np.fft.irfft2(Y, s=(fh, fw))
    valid = full[:, :, Rd - 1:Hp, Sd - 1:Wp]              # stride-1 correlation
    P = (H + 2 * ph - Rd) // u + 1
    Q = (W + 2 * pw - Sd) // v + 1
    y = valid[:, :, ::u, ::v][:, :, :P, :Q]
    if b is not None:
        y = y + b[None, :, None, None]
    return y


CASES = [
    # N, C, H, W, K, R, S, stride, pad, dil
    (1, 1, 5, 5, 1, 3, 3, (1, 1), (1, 1), (1, 1)),
    (2, 3, 7, 6, 4, 3, 3, (1, 1), (1, 1), (1, 1)),
    (2, 3, 9, 9, 2, 3, 3, (2, 2), (1, 1), (1, 1)),
    (1, 4, 9, 8, 3, 3, 2, (1, 2), (0, 1), (2, 1)),
    (2, 2, 8, 9, 3, 1, 1, (2, 1), (0, 0), (1, 1)),
    (1, 3, 9, 9, 2, 5, 5, (1, 1), (2, 2), (1, 1)),
    (1, 2, 9, 9, 2, 3, 3, (2, 2), (2, 2), (2, 2)),
    (2, 4, 6, 6, 4, 2, 2, (1, 1), (0, 1), (1, 1)),
]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_fft_bruteforce(case, layout):
    N, C, H, W, K, R, S, st, pd, dl = case
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, layout)
    r = _rng(hash(case) % 2**32)
    x = r.uniform(-1, 1, (N, C, H, W))
    w = r.uniform(-1, 1, (K, C, R, S))
    b = r.uniform(-0.1, 0.1, K)
    ref = _fft_conv(x, w, b, st, pd, dl)
    y = oracle.conv2d_fwd(p, _to_layout(x, layout), _to_layout(w, layout), b)
    y = _from_layout(y, layout)
    assert y.shape == ref.shape
    assert np.max(np.abs(y - ref)) < 1e-12


@pytest.mark.parametrize("case", CASES)
def test_torch_fp64_special_case(case):
    N, C, H, W, K, R, S, st, pd, dl = case
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, "NCHW")
    r = _rng(7)
    x = r.normal(size=(N, C, H, W))
    w = r.normal(size=(K, C, R, S))
    b = r.normal(size=K)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(w),
                                     torch.from_numpy(b), stride=st, padding=pd,
                                     dilation=dl).numpy()
    y = oracle.conv2d_fwd(p, x, w, b)
    assert np.max(np.abs(y - ref)) < 1e-11


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_identity_1x1(layout):
    N, C, H, W = 2, 5, 7, 6
    p = Conv(N, C, H, W, C, 1, 1, 1, 0, 1, layout)
    x = _rng(1).normal(size=(N, C, H, W))
    w = np.eye(C).reshape(C, C, 1, 1)
    y = oracle.conv2d_fwd(p, _to_layout(x, layout), _to_layout(w, layout))
    assert np.array_equal(_from_layout(y, layout), x)


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
@pytest.mark.parametrize("st,pd,dl,R,S", [
    ((1, 1), (1, 1), (1, 1), 3, 3),
    ((2, 2), (1, 1), (1, 1), 3, 3),
    ((1, 2), (2, 1), (2, 1), 3, 3),
    ((2, 1), (0, 3), (1, 3), 2, 3),
    ((1, 1), (3, 3), (1, 1), 7, 7),
])
def test_delta_filter_shift(layout, st, pd, dl, R, S):
    N, C, H, W = 2, 3, 9, 10
    r = _rng(2)
    x = r.normal(size=(N, C, H, W))
    for r0, s0 in itertools.product(range(R), range(S)):
        p = Conv(N, C, H, W, C, R, S, st, pd, dl, layout)
        w = np.zeros((C, C, R, S))
        for c in range(C):
            w[c, c, r0, s0] = 1.0
        y = _from_layout(oracle.conv2d_fwd(p, _to_layout(x, layout), _to_layout(w, layout)),
                         layout)
        # y[n,c,p,q] = x[n,c, p*u + r0*dh - ph, q*v + s0*dw - pw] (zero outside)
        exp = np.zeros((N, C, p.P, p.Q))
        for pp in range(p.P):
            for qq in range(p.Q):
                h = pp * st[0] + r0 * dl[0] - pd[0]
                ww = qq * st[1] + s0 * dl[1] - pd[1]
                if 0 <= h < H and 0 <= ww < W:
                    exp[:, :, pp, qq] = x[:, :, h, ww]
        assert np.array_equal(y, exp), (r0, s0)


def test_linearity():
    p = Conv(2, 3, 8, 8, 4, 3, 3, 1, 1, 1, "NHWC")
    r = _rng(3)
    x1, x2 = r.normal(size=p.x_shape), r.normal(size=p.x_shape)
    w1, w2 = r.normal(size=p.w_shape), r.normal(size=p.w_shape)
    a, b = 0.75, -2.5
    lhs = oracle.conv2d_fwd(p, a * x1 + b * x2, w1)
    rhs = a * oracle.conv2d_fwd(p, x1, w1) + b * oracle.conv2d_fwd(p, x2, w1)
    scale = np.max(np.abs(rhs))
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * scale
    lhs = oracle.conv2d_fwd(p, x1, a * w1 + b * w2)
    rhs = a * oracle.conv2d_fwd(p, x1, w1) + b * oracle.conv2d_fwd(p, x1, w2)
    assert np.max(np.abs(lhs - rhs)) < 1e-13 * scale


@pytest.mark.parametrize("case", CASES)
def test_integer_exact(case):
    """Integer inputs: every product and partial sum is an integer well below
    2^53, so the oracle's sum is exact and must equal the FFT result rounded
    to the nearest integer (FFT error << 0.5)."""
    N, C, H, W, K, R, S, st, pd, dl = case
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, "NCHW")
    r = _rng(4)
    x = r.integers(-4, 5, (N, C, H, W)).astype(np.float64)
    w = r.integers(-4, 5, (K, C, R, S)).astype(np.float64)
    b = r.integers(-8, 9, K).astype(np.float64)
    y = oracle.conv2d_fwd(p, x, w, b)
    ref = np.rint(_fft_conv(x, w, b, st, pd, dl))
    assert np.array_equal(y, ref)
    assert np.array_equal(y, np.rint(y))


def test_relu_and_bound():
    p = Conv(2, 3, 7, 7, 4, 3, 3, 1, 1, 1, "NHWC")
    r = _rng(5)
    x, w, b = r.normal(size=p.x_shape), r.normal(size=p.w_shape), r.normal(size=4)
    y, bound = oracle.conv2d_fwd(p, x, w, b, with_bound=True)
    yr = oracle.conv2d_fwd(p, x, w, b, relu=True)
    assert np.array_equal(yr, np.maximum(y, 0.0))
    assert np.all(np.abs(y) <= bound * (1 + 1e-15))
    # with non-negative x, w, b the bound is the sum itself
    y2, bound2 = oracle.conv2d_fwd(p, np.abs(x), np.abs(w), np.abs(b), with_bound=True)
    assert np.max(np.abs(y2 - bound2)) <= 1e-13 * np.max(bound2)


@pytest.mark.parametrize("case", CASES)
def test_adjoint_identities(case):
    N, C, H, W, K, R, S, st, pd, dl = case
    for layout in ("NCHW", "NHWC"):
        p = Conv(N, C, H, W, K, R, S, st, pd, dl, layout)
        r = _rng(6)
        x, w, g = r.normal(size=p.x_shape), r.normal(size=p.w_shape), r.normal(size=p.y_shape)
        y = oracle.conv2d_fwd(p, x, w)
        lhs = np.sum(y * g)
        dx = oracle.conv2d_dgrad(p, g, w)
        dw = oracle.conv2d_wgrad(p, x, g)
        scale = np.sum(np.abs(y * g)) + 1.0
        assert abs(lhs - np.sum(x * dx)) < 1e-12 * scale
        assert abs(lhs - np.sum(w * dw)) < 1e-12 * scale
        db = oracle.conv2d_bgrad(p, g)
        kax = 1 if layout == "NCHW" else 3
        axes = tuple(a for a in range(4) if a != kax)
        assert np.max(np.abs(db - g.sum(axis=axes))) < 1e-12 * (np.abs(g).sum() + 1)


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
@pytest.mark.parametrize("st,pd,dl", [((1, 1), (1, 1), (1, 1)), ((2, 2), (1, 1), (1, 1)),
                                      ((1, 2), (2, 0), (2, 1))])
def test_central_finite_differences(layout, st, pd, dl):
    """L = sum g*y is linear in each of x, w, b separately, so a central
    difference with a power-of-two step is exact up to roundoff. Size: N=1,
    C=K=4, H=W=6, 3x3 (the backward workload's tiny check)."""
    p = Conv(1, 4, 6, 6, 4, 3, 3, st, pd, dl, layout)
    r = _rng(8)
    x, w, b = r.normal(size=p.x_shape), r.normal(size=p.w_shape), r.normal(size=4)
    g = r.normal(size=p.y_shape)
    h = 2.0 ** -10

    def L(xx, ww, bb):
        return float(np.sum(oracle.conv2d_fwd(p, xx, ww, bb, nthreads=1) * g))

    def fd(arr, which):
        out = np.empty(arr.size)
        flat = arr.reshape(-1)
        for i in range(arr.size):
            keep = flat[i]
            flat[i] = keep + h
            lp = L(x, w, b)
            flat[i] = keep - h
            lm = L(x, w, b)
            flat[i] = keep
            out[i] = (lp - lm) / (2 * h)
        return out.reshape(arr.shape)

    dx_fd, dw_fd, db_fd = fd(x, "x"), fd(w, "w"), fd(b, "b")
    dx = oracle.conv2d_dgrad(p, g, w)
    dw = oracle.conv2d_wgrad(p, x, g)
    db = oracle.conv2d_bgrad(p, g)
    scale = np.sum(np.abs(g)) * max(np.max(np.abs(x)), np.max(np.abs(w)), 1.0)
    assert np.max(np.abs(dx - dx_fd)) < 1e-9 * scale
    assert np.max(np.abs(dw - dw_fd)) < 1e-9 * scale
    assert np.max(np.abs(db - db_fd)) < 1e-9 * scale


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_relu_gradient_central_differences(layout):
    """L = sum g * max(conv(x, w) + b, 0). With integer x, w and half-integer
    b every pre-activation z is k + 1/2, at least 1/2 away from the kink, and
    a step of 2^-10 in one element moves z by far less than that, so the
    central difference sees one linear piece and is exact up to roundoff. The
    chain rule through the oracle's relu_grad then gives dx, dw, db."""
    p = Conv(1, 4, 6, 6, 4, 3, 3, (1, 1), (1, 1), (1, 1), layout)
    r = _rng(18)
    x = r.integers(-3, 4, size=p.x_shape).astype(np.float64)
    w = r.integers(-3, 4, size=p.w_shape).astype(np.float64)
    b = r.integers(-4, 4, size=4).astype(np.float64) + 0.5
    g = r.normal(size=p.y_shape)
    h = 2.0 ** -10
    z = oracle.conv2d_fwd(p, x, w, b, nthreads=1)
    assert np.min(np.abs(z)) >= 0.5 and np.any(z < 0) and np.any(z > 0)
    y = oracle.conv2d_fwd(p, x, w, b, relu=True, nthreads=1)
    assert np.array_equal(y, np.maximum(z, 0.0))

    def L(xx, ww, bb):
        return float(np.sum(oracle.conv2d_fwd(p, xx, ww, bb, relu=True, nthreads=1) * g))

    def fd(arr):
        out = np.empty(arr.size)
        flat = arr.reshape(-1)
        for i in range(arr.size):
            keep = flat[i]
            flat[i] = keep + h
            lp = L(x, w, b)
            flat[i] = keep - h
            lm = L(x, w, b)
            flat[i] = keep
            out[i] = (lp - lm) / (2 * h)
        return out.reshape(arr.shape)

    gz = oracle.relu_grad(y, g)
    # a plausible slip (the mask from z >= 0, or no mask) changes the result
    assert not np.array_equal(gz, g)
    scale = np.sum(np.abs(g)) * max(np.max(np.abs(x)), np.max(np.abs(w)), 1.0)
    assert np.max(np.abs(oracle.conv2d_dgrad(p, gz, w) - fd(x))) < 1e-9 * scale
    assert np.max(np.abs(oracle.conv2d_wgrad(p, x, gz) - fd(w))) < 1e-9 * scale
    assert np.max(np.abs(oracle.conv2d_bgrad(p, gz) - fd(b))) < 1e-9 * scale


def test_relu_gradient_at_the_kink_and_signs():
    """Zero output (z <= 0) passes no gradient, positive output passes it
    unchanged, whatever the sign of g; -0.0 counts as zero."""
    y = np.array([0.0, -0.0, 1e-300, 2.5, -3.0, 0.0])
    g = np.array([1.0, -2.0, 3.0, -4.0, 5.0, -6.0])
    assert np.array_equal(oracle.relu_grad(y, g), np.array([0.0, 0.0, 3.0, -4.0, 0.0, 0.0]))


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_points_equal_full(layout):
    p = Conv(2, 5, 9, 7, 6, 3, 3, (2, 1), (1, 1), (1, 2), layout)
    r = _rng(9)
    x, w, b = r.normal(size=p.x_shape), r.normal(size=p.w_shape), r.normal(size=6)
    g = r.normal(size=p.y_shape)
    y, yb = oracle.conv2d_fwd(p, x, w, b, relu=True, with_bound=True)
    idx = r.choice(y.size, 50, replace=False)
    yp, ypb = oracle.conv2d_fwd(p, x, w, b, relu=True, idx=idx, with_bound=True)
    assert np.array_equal(yp, y.reshape(-1)[idx]) and np.array_equal(ypb, yb.reshape(-1)[idx])
    dx = oracle.conv2d_dgrad(p, g, w)
    idx = r.choice(dx.size, 50, replace=False)
    assert np.array_equal(oracle.conv2d_dgrad(p, g, w, idx=idx), dx.reshape(-1)[idx])
    dw = oracle.conv2d_wgrad(p, x, g)
    idx = r.choice(dw.size, 50, replace=False)
    assert np.array_equal(oracle.conv2d_wgrad(p, x, g, idx=idx), dw.reshape(-1)[idx])


def test_layouts_agree():
    p0 = Conv(2, 3, 8, 7, 5, 3, 2, (1, 2), (1, 0), (2, 1), "NCHW")
    p1 = Conv(2, 3, 8, 7, 5, 3, 2, (1, 2), (1, 0), (2, 1), "NHWC")
    r = _rng(10)
    x, w, b = r.normal(size=p0.x_shape), r.normal(size=p0.w_shape), r.normal(size=5)
    y0 = oracle.conv2d_fwd(p0, x, w, b)
    y1 = oracle.conv2d_fwd(p1, _to_layout(x, "NHWC"), _to_layout(w, "NHWC"), b)
    assert np.array_equal(y0, _from_layout(y1, "NHWC"))


def test_output_dims():
    for (H, R, pad, dil, st) in [(56, 3, 1, 1, 2), (56, 1, 0, 1, 1), (7, 7, 3, 1, 2),
                                 (112, 5, 2, 1, 2), (32, 3, 1, 1, 1), (6, 3, 0, 2, 1)]:
        p = Conv(1, 1, H, H, 1, R, R, st, pad, dil)
        ref = torch.nn.functional.conv2d(torch.zeros(1, 1, H, H), torch.zeros(1, 1, R, R),
                                         stride=st, padding=pad, dilation=dil).shape[2]
        assert p.P == ref and p.Q == ref
    with pytest.raises(ValueError):
        Conv(1, 1, 2, 2, 1, 5, 5, 1, 0, 1)


# ---- quantisers ----

def test_bf16_rounding_matches_definition_and_torch():
    r = _rng(11)
    vals = np.concatenate([
        r.normal(size=20000).astype(np.float32),
        (r.normal(size=2000) * 1e-39).astype(np.float32),          # subnormals
        np.array([0.0, -0.0, 1.0, -1.0, 3.4e38, -3.4e38, np.inf, -np.inf], np.float32),
    ])
    # exact ties: values halfway between two bf16 neighbours
    base = r.integers(0, 0x7F80, 1000).astype(np.uint32) << 16    # finite patterns
    ties = (base | 0x8000).view(np.float32)
    vals = np.concatenate([vals, ties])
    got = oracle.round_bf16_bits(vals)
    ref = torch.from_numpy(vals).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(got, ref)
    # ties go to the even neighbour
    tb = oracle.round_bf16_bits(ties)
    assert np.all((tb & 1) == 0)
    # nan stays nan
    assert np.isnan(oracle.round_bf16(np.array([np.nan], np.float32)))[0]


def test_e4m3_codes_roundtrip():
    codes = np.arange(256, dtype=np.uint8)
    vals = oracle.e4m3_to_f64(codes)
    nan = (codes & 0x7F) == 0x7F
    assert np.all(np.isnan(vals[nan])) and not np.any(np.isnan(vals[~nan]))
    assert np.max(vals[~nan]) == 448.0 and np.min(vals[~nan]) == -448.0
    assert vals[1] == 2.0 ** -9                      # smallest subnormal
    assert vals[0x08] == 2.0 ** -6                   # smallest normal
    back = oracle.quant_e4m3(vals[~nan].astype(np.float32))
    assert np.array_equal(back, codes[~nan])
    # decoding agrees with torch's float8_e4m3fn interpretation of the same bits
    tv = torch.from_numpy(codes[~nan].copy()).view(torch.float8_e4m3fn).to(torch.float64)
    assert np.array_equal(tv.numpy(), vals[~nan])


def test_e4m3_rounding_ties_and_saturation():
    codes = np.arange(0, 0x7E, dtype=np.uint8)      # positive finite codes, ascending
    v = oracle.e4m3_to_f64(np.arange(0, 0x7F, dtype=np.uint8))
    mids = ((v[:-1] + v[1:]) / 2).astype(np.float32)
    assert np.array_equal(mids.astype(np.float64), (v[:-1] + v[1:]) / 2)  # exact in fp32
    got = oracle.quant_e4m3(mids)
    lo, hi = codes, codes + 1
    want = np.where(lo % 2 == 0, lo, hi).astype(np.uint8)
    assert np.array_equal(got, want)
    big = np.array([448.0, 449.0, 463.9, 464.0, 1e6, np.float32(3e38)], np.float32)
    assert np.all(oracle.quant_e4m3(big) == 0x7E)
    assert np.all(oracle.quant_e4m3(-big) == 0xFE)


def test_e4m3_matches_torch_within_range():
    r = _rng(12)
    vals = np.concatenate([r.normal(size=50000) * 60, r.normal(size=5000) * 1e-2,
                           r.normal(size=5000) * 1e-3]).astype(np.float32)
    vals = np.clip(vals, -448, 448)
    got = oracle.e4m3_to_f64(oracle.quant_e4m3(vals))
    ref = torch.from_numpy(vals).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(got, ref)


def test_scale_quant_definition():
    r = _rng(13)
    a = (r.normal(size=(6, 300)) * r.uniform(0.01, 10, (6, 1))).astype(np.float32)
    a[2] = 0.0
    codes, scales = oracle.scale_quant_e4m3(a, 6)
    amax = np.max(np.abs(a), axis=1)
    want = np.maximum((amax / np.float32(448.0)).astype(np.float32), np.float32(1e-12))
    assert np.array_equal(scales, want)
    vals = oracle.e4m3_to_f64(codes)
    # the largest-magnitude element of each row lands on +-448 (or near it)
    for i in range(6):
        if amax[i] > 0:
            assert np.max(np.abs(vals[i])) >= 416.0
    assert np.all(vals[2] == 0)
    # dequantised values are close to the input (3 mantissa bits: rel err <= 2^-4)
    deq = vals * scales[:, None]
    big = np.abs(a) > scales[:, None] * 2.0 ** -6 * 4
    assert np.all(np.abs(deq - a)[big] <= np.abs(a)[big] * 2.0 ** -4 * (1 + 1e-6))


# ---- fused forward (batch normalisation folded, residual add, ReLU) ----

@pytest.mark.parametrize("case", CASES[:6])
@pytest.mark.parametrize("relu", [False, True])
def test_fused_bn_residual_matches_torch_library(case, relu):
    """conv + bias -> inference batch_norm -> + residual -> ReLU with PyTorch's
    own float64 conv2d and batch_norm equals the oracle's fused forward with
    the folded (alpha, beta): pins the fold formula, where alpha and beta enter,
    the residual's indexing and the activation."""
    N, C, H, W, K, R, S, st, pd, dl = case
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, "NCHW")
    r = _rng(11)
    x = r.normal(size=(N, C, H, W))
    w = r.normal(size=(K, C, R, S))
    b = r.normal(size=K)
    gamma, bn_beta = r.uniform(0.5, 1.5, K), r.normal(size=K)
    mean, var, eps = r.normal(size=K), r.uniform(0.2, 2.0, K), 1e-5
    z = r.normal(size=p.y_shape)
    T = torch.from_numpy
    ref = torch.nn.functional.conv2d(T(x), T(w), T(b), stride=st, padding=pd, dilation=dl)
    ref = torch.nn.functional.batch_norm(ref, T(mean), T(var), T(gamma), T(bn_beta),
                                         training=False, eps=eps) + T(z)
    if relu:
        ref = torch.relu(ref)
    alpha, beta = oracle.bn_fold(gamma, bn_beta, mean, var, eps, bias=b)
    y = oracle.conv2d_fwd_fused(p, x, w, alpha, beta, z, relu=relu)
    assert np.max(np.abs(y - ref.numpy())) < 1e-10


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_fused_defaults_reduce_to_plain_forward(layout):
    p = Conv(2, 3, 7, 6, 4, 3, 3, (1, 1), (1, 1), (1, 1), layout)
    r = _rng(12)
    x, w, b = r.normal(size=p.x_shape), r.normal(size=p.w_shape), r.normal(size=4)
    y0, b0 = oracle.conv2d_fwd(p, x, w, b, relu=True, with_bound=True)
    y1, b1 = oracle.conv2d_fwd_fused(p, x, w, None, b, None, relu=True, with_bound=True)
    assert np.array_equal(y0, y1) and np.array_equal(b0, b1)


@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_fused_integer_residual_and_power_of_two_scale_exact(layout):
    """Integer operands, alpha a power of two: every step is exact in FP64, so
    y = 4*conv + beta + z holds bit for bit, and the bound adds |alpha|, |beta|
    and |z| the same way."""
    p = Conv(2, 4, 6, 7, 3, 3, 3, (2, 1), (1, 1), (1, 1), layout)
    r = _rng(13)
    x = r.integers(-4, 5, p.x_shape).astype(float)
    w = r.integers(-4, 5, p.w_shape).astype(float)
    beta = r.integers(-8, 9, 3).astype(float)
    z = r.integers(-16, 17, p.y_shape).astype(float)
    alpha = np.full(3, -4.0)
    y, bound = oracle.conv2d_fwd_fused(p, x, w, alpha, beta, z, with_bound=True)
    c, cb = oracle.conv2d_fwd(p, x, w, None, with_bound=True)
    kax = 1 if layout == "NCHW" else 3
    shape = [1, 1, 1, 1]
    shape[kax] = 3
    assert np.array_equal(y, -4.0 * c + beta.reshape(shape) + z)
    assert np.array_equal(bound, 4.0 * cb + np.abs(beta).reshape(shape) + np.abs(z))


def test_bn_fold_definition():
    """alpha*(conv + b) normalised and shifted equals alpha*conv + beta for any
    conv value: checked at random points against the unfolded formula."""
    r = _rng(14)
    K = 9
    gamma, bn_beta, b = r.normal(size=K), r.normal(size=K), r.normal(size=K)
    mean, var, eps = r.normal(size=K), r.uniform(0.1, 3, K), 1e-3
    alpha, beta = oracle.bn_fold(gamma, bn_beta, mean, var, eps, bias=b)
    for v in r.normal(size=5) * 10:
        unfolded = (v + b - mean) / np.sqrt(var + eps) * gamma + bn_beta
        assert np.max(np.abs(alpha * v + beta - unfolded)) < 1e-12
    a0, b0 = oracle.bn_fold(gamma, bn_beta, mean, var, eps)
    assert np.allclose(b0, bn_beta - mean * a0, rtol=0, atol=1e-15)


# ---- channel groups (G = C = K: depthwise) ----

GROUP_CASES = [
    # N, C, H, W, K, R, S, stride, pad, dil, G
    (2, 4, 7, 6, 6, 3, 3, (1, 1), (1, 1), (1, 1), 2),
    (1, 8, 9, 9, 8, 3, 3, (2, 2), (1, 1), (1, 1), 8),     # depthwise
    (2, 6, 8, 7, 12, 3, 2, (1, 2), (1, 0), (2, 1), 6),    # depthwise, multiplier 2
    (1, 12, 9, 8, 8, 5, 5, (1, 1), (2, 2), (1, 1), 4),
    (2, 16, 6, 6, 16, 1, 1, (1, 1), (0, 0), (1, 1), 16),  # 1x1 depthwise: a per-channel scale
]


@pytest.mark.parametrize("case", GROUP_CASES)
@pytest.mark.parametrize("layout", ["NCHW", "NHWC"])
def test_groups_match_torch_library(case, layout):
    """Forward, data and weight gradients with channel groups against PyTorch's
    float64 conv2d(groups=G) and its autograd."""
    N, C, H, W, K, R, S, st, pd, dl, G = case
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, layout, groups=G)
    r = _rng(21)
    x = torch.from_numpy(r.normal(size=(N, C, H, W))).requires_grad_()
    w = torch.from_numpy(r.normal(size=(K, C // G, R, S))).requires_grad_()
    b = torch.from_numpy(r.normal(size=K))
    y = torch.nn.functional.conv2d(x, w, b, stride=st, padding=pd, dilation=dl, groups=G)
    g = torch.from_numpy(r.normal(size=tuple(y.shape)))
    (y * g).sum().backward()
    yo = oracle.conv2d_fwd(p, _to_layout(x.detach().numpy(), layout),
                           _to_layout(w.detach().numpy(), layout), b.numpy())
    assert np.max(np.abs(_from_layout(yo, layout) - y.detach().numpy())) < 1e-11
    go = _to_layout(g.numpy(), layout)
    dx = oracle.conv2d_dgrad(p, go, _to_layout(w.detach().numpy(), layout))
    dw = oracle.conv2d_wgrad(p, _to_layout(x.detach().numpy(), layout), go)
    assert np.max(np.abs(_from_layout(dx, layout) - x.grad.numpy())) < 1e-11
    assert np.max(np.abs(_from_layout(dw, layout) - w.grad.numpy())) < 1e-10


@pytest.mark.parametrize("case", GROUP_CASES[:4])
def test_groups_are_independent_convolutions(case):
    """Output channels of group g equal an ungrouped convolution of x's channel
    slice g with the filters of group g (exact: the same sum in the same order)."""
    N, C, H, W, K, R, S, st, pd, dl, G = case
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, "NCHW", groups=G)
    r = _rng(22)
    x, w, b = r.normal(size=(N, C, H, W)), r.normal(size=(K, C // G, R, S)), r.normal(size=K)
    y = oracle.conv2d_fwd(p, x, w, b)
    cg, kg = C // G, K // G
    for g in range(G):
        pg = Conv(N, cg, H, W, kg, R, S, st, pd, dl, "NCHW")
        yg = oracle.conv2d_fwd(pg, np.ascontiguousarray(x[:, g * cg:(g + 1) * cg]),
                               np.ascontiguousarray(w[g * kg:(g + 1) * kg]), b[g * kg:(g + 1) * kg])
        assert np.array_equal(y[:, g * kg:(g + 1) * kg], yg)


def test_groups_adjoint_identities():
    N, C, H, W, K, R, S, st, pd, dl, G = GROUP_CASES[2]
    p = Conv(N, C, H, W, K, R, S, st, pd, dl, "NHWC", groups=G)
    r = _rng(23)
    x, w = r.normal(size=p.x_shape), r.normal(size=p.w_shape)
    g = r.normal(size=p.y_shape)
    lhs = np.sum(oracle.conv2d_fwd(p, x, w) * g)
    assert abs(lhs - np.sum(x * oracle.conv2d_dgrad(p, g, w))) < 1e-9 * max(1, abs(lhs))
    assert abs(lhs - np.sum(w * oracle.conv2d_wgrad(p, x, g))) < 1e-9 * max(1, abs(lhs))


def test_groups_must_divide_channels():
    with pytest.raises(ValueError):
        Conv(1, 6, 5, 5, 4, 3, 3, groups=4)


# ---- negative log-likelihood loss ----

@pytest.mark.parametrize("reduction", ["none", "mean", "sum"])
@pytest.mark.parametrize("weighted", [False, True])
def test_nll_loss_matches_torch_library(reduction, weighted):
    """Forward and gradient against PyTorch's float64 nll_loss and its autograd,
    with ignored rows."""
    r = _rng(31)
    N, C = 37, 11
    logp = torch.log_softmax(torch.from_numpy(r.normal(size=(N, C))), dim=1).requires_grad_()
    t = torch.from_numpy(r.integers(0, C, N))
    t[[3, 10, 20]] = -100
    w = torch.from_numpy(r.uniform(0.5, 2.0, C)) if weighted else None
    ref = torch.nn.functional.nll_loss(logp, t, weight=w, ignore_index=-100, reduction=reduction)
    g = torch.from_numpy(r.normal(size=tuple(ref.shape)))
    (ref * g).sum().backward()
    out, tw = oracle.nll_loss(logp.detach().numpy(), t.numpy(), w.numpy() if weighted else None,
                              -100, reduction)
    assert np.max(np.abs(out.reshape(ref.shape) - ref.detach().numpy())) < 1e-12
    gi = oracle.nll_loss_grad(g.numpy(), t.numpy(), N, C, w.numpy() if weighted else None, -100,
                              reduction, tw)
    assert np.max(np.abs(gi - logp.grad.numpy())) < 1e-12


def test_nll_loss_worked_example():
    """Two rows, three classes, by hand: -(log 0.5 + 2 log 0.25) / (1 + 2)."""
    logp = np.log(np.array([[0.5, 0.25, 0.25], [0.25, 0.25, 0.5]]))
    out, tw = oracle.nll_loss(logp, [0, 1], weight=[1.0, 2.0, 3.0], reduction="mean")
    assert tw == 3.0 and abs(out[0] - (-(np.log(0.5) + 2 * np.log(0.25)) / 3)) < 1e-15
    gi = oracle.nll_loss_grad([1.0], [0, 1], 2, 3, [1.0, 2.0, 3.0], reduction="mean",
                              total_weight=tw)
    assert np.array_equal(gi, np.array([[-1 / 3, 0, 0], [0, -2 / 3, 0]]))


def test_nll_loss_rejects_bad_targets():
    with pytest.raises(ValueError):
        oracle.nll_loss(np.zeros((2, 3)), [0, 3])
