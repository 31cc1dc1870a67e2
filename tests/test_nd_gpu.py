"""GPU parity of multidimensional convolutions (Section 5 decomposition:
outer-axis residue transforms, inner sub-convolutions, inverse outer
transforms) against the FP64 direct N-D oracle."""
import itertools

import numpy as np
import pytest

import inputs
from oracle import direct, explicit, params
from tests.gpu_util import rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hd():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2303_17510_gb300 as hd
    return hd


def run_nd(hd, plan, fs, dtype):
    import torch
    d = [to_dev(f, dtype) for f in fs]
    out = torch.zeros_like(d[0])
    plan.convolve(d, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def axis_kinds(kind, nd):
    outer = "complex" if kind == "complex" else "centered"
    return tuple([outer] * (nd - 1) + [kind])


def bounds(kind, shape_L, mult="product"):
    ks = axis_kinds(kind, len(shape_L))
    return [params.dealias_bound(k, L, mult) for k, L in zip(ks, shape_L)]


def make_nd(kind, Ls, A, seed, integer=False):
    gen = inputs.integer_complex if integer else inputs.uniform_complex
    return [gen(tuple(Ls), seed + a) for a in range(A)]


@pytest.mark.parametrize("kind", ["complex", "centered"])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("Ls", [(5, 7), (16, 12), (31, 33), (6, 5, 7)])
def test_nd_small_matches_oracle(hd, kind, dtype, Ls):
    fs = make_nd(kind, Ls, 2, 10 + sum(Ls), integer=(dtype == "f64"))
    ref = direct.convnd(fs, axis_kinds(kind, len(Ls)))
    Ms = [b + 1 for b in bounds(kind, Ls)]
    with hd.Plan(list(Ls), Ms, kind=kind, dtype=dtype) as plan:
        got = run_nd(hd, plan, fs, dtype)
    if dtype == "f64":
        assert np.array_equal(np.rint(got.real) + 1j * np.rint(got.imag), ref)
    else:
        assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_nd_hermitian_small(hd, dtype):
    L = 12
    fs = [inputs.hermitian_3d(L, 40 + a, dtype=np.complex128) for a in range(2)]
    ref = direct.convnd(fs, ("centered", "centered", "hermitian"))
    Ms = [b + 2 for b in bounds("hermitian", (L, L, L))]
    with hd.Plan([L, L, L], Ms, kind="hermitian", dtype=dtype) as plan:
        got = run_nd(hd, plan, fs, dtype)
    assert rel_l2(got, ref) <= (1e-5 if dtype == "f32" else 1e-12)


def test_nd_sum_pairs3_and_explicit_parameters(hd):
    Ls = (20, 24)
    fs = make_nd("complex", Ls, 3, 77)
    ref = direct.convnd(fs, ("complex", "complex"), "sum_pairs3")
    Ms = bounds("complex", Ls, "sum_pairs3")
    # every legal m of the outer axis, with residues one at a time (D = 1) or all at once
    for mx in (4, 8, 16, 32, 64):
        for D in (0, 1):
            try:
                plan = hd.Plan(list(Ls), Ms, A=3, m=[mx, 0], D=[D, 0])
            except hd.HdError as e:
                assert e.name == "HD_ERR_UNSUPPORTED"
                continue
            with plan:
                got = run_nd(hd, plan, fs, "f32")
                assert rel_l2(got, ref) <= 1e-5, (mx, D, plan.axis_params(0))


U32 = 2.0 ** -24      # unit roundoff of FP32


def field_checks(got, want, Ntotal, tile):
    """Whole-field comparison of an FP32 result with the FP64 oracle.

    FFT rounding errors spread over the data a transform mixes, at about u
    log2(N) times its RMS magnitude (u the FP32 unit roundoff, N the transform
    size); values far below that level cannot be resolved.  A multi-axis
    decomposition transforms lines of very different norms (a decaying
    spectrum concentrates its magnitude near k = 0), and the outer inverse
    transforms spread the rounding errors of the innermost-axis convolutions
    over the whole hyperplane of fixed innermost index, so the level varies
    over the field.  Three checks: rel-L2 over the field <= 1e-5; per tile of
    the given shape, RMS error <= 1e-5 of the tile's RMS output plus 2 u
    log2(N) of the global RMS; per point, error <= 1e-5 of the point's
    magnitude plus 10 u log2(N) of the largest of the global RMS, the RMS of
    the point's tile and the RMS of its hyperplane.  A wrong region fails the
    tile check unless its exact values are themselves below the rounding level
    of the transform."""
    got = np.asarray(got, dtype=np.complex128)
    want = np.asarray(want, dtype=np.complex128)
    assert got.shape == want.shape
    err = np.abs(got - want)
    rms = float(np.sqrt(np.mean(np.abs(want) ** 2)))
    level = U32 * np.log2(Ntotal)
    stats = {"rel_l2": rel_l2(got, want)}
    assert stats["rel_l2"] <= 1e-5, stats
    shp = [s // t for s, t in zip(want.shape, tile)]
    full = tuple(slice(0, s * t) for s, t in zip(shp, tile))
    blk = lambda x: x[full].reshape([v for pair in zip(shp, tile) for v in pair])
    axes = tuple(range(1, 2 * len(tile), 2))
    e_t = np.sqrt(np.mean(blk(err) ** 2, axis=axes))
    w_t = np.sqrt(np.mean(blk(np.abs(want)) ** 2, axis=axes))
    stats["tile_excess"] = float(np.max(e_t / (1e-5 * w_t + 2 * level * rms)))
    assert stats["tile_excess"] <= 1.0, stats
    # the RMS of each point's tile, broadcast back to the points
    w_pt = w_t
    for ax, t in enumerate(tile):
        w_pt = np.repeat(w_pt, t, axis=ax)
    # RMS of each hyperplane of fixed innermost index, broadcast to the points
    w_pl = np.sqrt(np.mean(np.abs(want) ** 2, axis=tuple(range(want.ndim - 1)), keepdims=True))
    local = np.maximum(np.maximum(rms, w_pt), np.broadcast_to(w_pl, want.shape)[full])
    ratio = err[full] / (1e-5 * np.abs(want[full]) + 10 * level * local)
    stats["point_excess"] = float(np.max(ratio))
    if stats["point_excess"] > 1.0:
        j = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
        stats.update(worst=tuple(int(x) for x in j), err=float(err[j]), want=float(np.abs(want[j])),
                     tile_rms=float(w_pt[j]), plane_rms=float(w_pl.ravel()[j[-1]]), rms=rms)
    assert stats["point_excess"] <= 1.0, "; ".join(f"{k}={v}" for k, v in stats.items())
    return stats


def point_checks(got, want, Ntotal, rms):
    """Exact oracle points (direct sums): rel-L2 over the points <= 1e-5 and
    the per-point bound of field_checks."""
    assert rel_l2(got, want) <= 1e-5
    noise = U32 * np.log2(Ntotal) * rms
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 10 * noise)


def test_2d_full_size(hd):
    """2048 x 2048 complex, M = 4095 per axis, spectrum (1+|k|)^-1 (the 2D
    workload): the whole field against the FP64 explicit zero-padded FFT
    convolution on 4096^2, and 256 + 4 points against the exact direct sum."""
    L = 2048
    fs = [inputs.spectral_2d(L, L, 3 + a, dtype=np.complex64) for a in range(2)]
    with hd.Plan([L, L], [2 * L - 1, 2 * L - 1]) as plan:
        got = run_nd(hd, plan, fs, "f32")
        Ntot = 1
        for i in range(2):
            ax = plan.axis_params(i)
            Ntot *= ax["n"] * ax["S"]
    f64 = [f.astype(np.complex128) for f in fs]
    full = explicit.convnd_explicit(f64, ("complex", "complex"), [4096, 4096])
    field_checks(got, full, Ntot, (64, 64))
    rng = np.random.default_rng(0)
    pts = np.stack([rng.integers(0, L, 256), rng.integers(0, L, 256)], axis=1)
    pts = np.concatenate([pts, [[0, 0], [L - 1, L - 1], [0, L - 1], [L - 1, 0]]])
    want = direct.convnd_points(f64, ("complex", "complex"), pts)
    assert np.allclose(full[tuple(pts.T)], want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))
    point_checks(got[tuple(pts.T)], want, Ntot, float(np.sqrt(np.mean(np.abs(full) ** 2))))


def test_3d_hermitian_full_size(hd):
    """256^3 centered Hermitian (128 stored on the last axis), M = 384 per
    axis: the whole stored field against the FP64 explicit zero-padded FFT
    convolution of the expanded Hermitian array on 384^3, and 256 + 3 points
    against the exact direct sum."""
    L = 256
    fs = [inputs.hermitian_3d(L, 5 + a, dtype=np.complex64) for a in range(2)]
    kinds = ("centered", "centered", "hermitian")
    with hd.Plan([L, L, L], [384, 384, 384], kind="hermitian") as plan:
        got = run_nd(hd, plan, fs, "f32")
        Ntot = 1
        for i in range(3):
            ax = plan.axis_params(i)
            Ntot *= ax["n"] * ax["S"]
    f64 = [f.astype(np.complex128) for f in fs]
    full = explicit.convnd_explicit(f64, kinds, [384, 384, 384])
    field_checks(got, full, Ntot, (32, 32, 16))
    rng = np.random.default_rng(1)
    H = L // 2
    pts = np.stack([rng.integers(0, L, 256), rng.integers(0, L, 256), rng.integers(0, H, 256)], axis=1)
    pts = np.concatenate([pts, [[L // 2, L // 2, 0], [0, 0, 0], [L - 1, L - 1, H - 1]]])
    want = direct.convnd_points(f64, kinds, pts)
    assert np.allclose(full[tuple(pts.T)], want, rtol=1e-12, atol=1e-12 * np.max(np.abs(want)))
    point_checks(got[tuple(pts.T)], want, Ntot, float(np.sqrt(np.mean(np.abs(full) ** 2))))


@pytest.mark.parametrize("kind", ["complex", "hermitian"])
def test_3d_middle_level_chunks(hd, monkeypatch, kind):
    """The middle axis of a 3D plan can run its independent instances (the
    outer axis's transformed slices) in chunks whose work buffer stays in L2
    (HD_ND_CHUNK_MB; off by default): a small chunk limit gives the same
    result, bit for bit, as no limit, and the FP32 bound against the FP64
    explicit zero-padded FFT convolution."""
    L = 40
    if kind == "hermitian":
        fs = [inputs.hermitian_3d(L, 770 + a, dtype=np.complex64) for a in range(2)]
        kinds, Ms = ("centered", "centered", "hermitian"), [60, 60, 60]
    else:
        fs = [inputs.uniform_complex((L, L, L), 770 + a, dtype=np.complex64) for a in range(2)]
        kinds, Ms = ("complex",) * 3, [79, 79, 79]
    outs = []
    for mb in ("1", ""):
        monkeypatch.setenv("HD_ND_CHUNK_MB", mb)
        with hd.Plan([L, L, L], Ms, kind=kind) as plan:
            outs.append(run_nd(hd, plan, fs, "f32"))
    assert np.array_equal(outs[0], outs[1])
    want = explicit.convnd_explicit([f.astype(np.complex128) for f in fs], kinds, Ms)
    assert rel_l2(outs[0], want) <= 1e-5
