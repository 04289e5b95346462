"""The autotuner of the tcgen05 column tile (and, for the batched solver, of the product schedule:
one CTA per work item or a persistent CTA per SM): its choices are cached per context, persist through
the TSTAR_TUNE_CACHE file, and do not change results (every output entry accumulates the same
products in the same order whatever the tile width or schedule)."""
import numpy as np
import pytest

from oracle import krylov as kr
from paper_2405_09233_gb300 import inputs
from tests.gpu_helpers import to_dev, from_dev

pytestmark = pytest.mark.gpu

PREC_CODE = {"mixed_tf32": 2, "mixed_bf16": 3, "mixed_tf32x3": 4}


def _apply(ctx, shape, prec):
    import torch
    n, s, p = shape
    pr = inputs.dense_problem(n, s, p, seed=11 + n)
    X32 = inputs.random_tensor((n, s, p), seed=12).astype(np.float32)
    op = ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B))
    Y = from_dev(ctx.sylv_apply_lowp(op, torch.from_numpy(inputs.to_device_layout(X32)).cuda(), prec))
    op.close()
    return Y


def _key(shape, prec):
    n, s, p = shape
    return f"tc:{n}x{s}x{p // 2 + 1}:{PREC_CODE[prec]}"


def _lines(path):
    return [ln for ln in path.read_text().splitlines() if ln.strip()] if path.exists() else []


def test_choice_cached_and_persisted(tmp_path, monkeypatch):
    from paper_2405_09233_gb300 import Context
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("TSTAR_TUNE_CACHE", str(cache))
    shape, prec = (300, 200, 8), "mixed_bf16"
    with Context(0) as ctx:
        _apply(ctx, shape, prec)
        ent = ctx.tune_entries()
        assert ent[_key(shape, prec)] in (64, 128, 256)
        lines = _lines(cache)
        assert len(lines) == 1 and lines[0].split()[1:] == [_key(shape, prec), str(ent[_key(shape, prec)])]
        _apply(ctx, shape, prec)                          # cached in the context: nothing retimed
        assert len(_lines(cache)) == 1
    with Context(0) as ctx:                               # a new context reads the file
        _apply(ctx, shape, prec)
        assert ctx.tune_entries()[_key(shape, prec)] == int(lines[0].split()[2])
        assert len(_lines(cache)) == 1


def _device_tag(tmp_path, monkeypatch):
    from paper_2405_09233_gb300 import Context
    probe = tmp_path / "probe.txt"
    monkeypatch.setenv("TSTAR_TUNE_CACHE", str(probe))
    with Context(0) as ctx:
        _apply(ctx, (64, 200, 2), "mixed_bf16")
    return _lines(probe)[0].split()[0]


@pytest.mark.parametrize("prec", ["mixed_bf16", "mixed_tf32x3"])
def test_tile_width_does_not_change_result(tmp_path, monkeypatch, prec):
    """Force each candidate width through the cache file: the products agree bit for bit."""
    from paper_2405_09233_gb300 import Context
    tag = _device_tag(tmp_path, monkeypatch)
    shape = (200, 300, 6)                                 # ragged in both tile directions
    outs = {}
    for bn in (64, 128, 256):
        cache = tmp_path / f"forced_{bn}.txt"
        cache.write_text(f"{tag} {_key(shape, prec)} {bn}\n")
        monkeypatch.setenv("TSTAR_TUNE_CACHE", str(cache))
        with Context(0) as ctx:
            outs[bn] = _apply(ctx, shape, prec)
            assert ctx.tune_entries()[_key(shape, prec)] == bn
        assert len(_lines(cache)) == 1                    # nothing was tuned
    assert np.isfinite(outs[64]).all()
    for bn in (128, 256):
        assert np.array_equal(outs[64].view(np.uint32), outs[bn].view(np.uint32)), bn


def test_malformed_cache_lines_ignored(tmp_path, monkeypatch):
    from paper_2405_09233_gb300 import Context
    tag = _device_tag(tmp_path, monkeypatch)
    shape, prec = (130, 70, 8), "mixed_tf32"
    cache = tmp_path / "bad.txt"
    cache.write_text("garbage\n\n"
                     f"{tag} {_key(shape, prec)} notanumber\n"
                     f"other_device {_key(shape, prec)} 64\n"
                     f"{tag} {_key(shape, prec)} 96\n")       # not a candidate: tuned afresh
    monkeypatch.setenv("TSTAR_TUNE_CACHE", str(cache))
    with Context(0) as ctx:
        _apply(ctx, shape, prec)
        assert ctx.tune_entries()[_key(shape, prec)] in (64, 128)
    assert _lines(cache)[-1].split()[:2] == [tag, _key(shape, prec)]


def test_batched_tile_tuned(tmp_path, monkeypatch):
    import torch
    from paper_2405_09233_gb300 import Context
    monkeypatch.setenv("TSTAR_TUNE_CACHE", str(tmp_path / "b.txt"))
    shapes = [(96, 40, 4), (130, 150, 8), (64, 64, 2)]
    with Context(0) as ctx:
        ops, Cs, Xs = [], [], []
        for i, (n, s, p) in enumerate(shapes):
            pr = inputs.dense_problem(n, s, p, seed=40 + i)
            ops.append(ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B)))
            Cs.append(to_dev(kr.sylv_apply(pr.A, pr.B, pr.Xstar)))
            Xs.append(torch.zeros((p, s, n), dtype=torch.float64, device="cuda"))
        st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=20, precision="mixed_bf16", engine="ozaki")
        assert st == 0 and all(x == 0 for x in sts)
        btc = [v for k, v in ctx.tune_entries().items() if k.startswith("btc:")]
        assert len(btc) == 1 and btc[0] in (64, 65, 128, 129)   # column tile, + 1 when persistent
        for op in ops:
            op.close()


@pytest.mark.parametrize("prec", ["mixed_bf16", "mixed_tf32x3"])
def test_batched_schedules_agree_bitwise(tmp_path, monkeypatch, prec):
    """Force each batched product schedule (column tile 64 or 128, one CTA per work item or the persistent
    kernel walking the work list) through the cache file: the batched solves agree bit for bit."""
    import torch
    from paper_2405_09233_gb300 import Context
    tag = _device_tag(tmp_path, monkeypatch)
    shapes = [(96, 40, 4), (130, 150, 8), (64, 64, 2), (200, 90, 6)]   # ragged tiles, real and complex slices
    key = f"btc:{PREC_CODE[prec]}:{len(shapes)}" + "".join(f":{n}x{s}x{p // 2 + 1}" for n, s, p in shapes)
    probs = [inputs.dense_problem(n, s, p, seed=60 + i) for i, (n, s, p) in enumerate(shapes)]
    Cs_h = [kr.sylv_apply(pr.A, pr.B, pr.Xstar) for pr in probs]
    outs = {}
    simt = f"bsimt:8:{len(shapes)}" + "".join(f":{n}x{s}x{p // 2 + 1}" for n, s, p in shapes)
    for sched in (64, 65, 128, 129):
        cache = tmp_path / f"b_{sched}.txt"
        cache.write_text(f"{tag} {key} {sched}\n{tag} {simt} 64\n")   # and the FP64 residual products' tile
        monkeypatch.setenv("TSTAR_TUNE_CACHE", str(cache))
        with Context(0) as ctx:
            ops = [ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B)) for pr in probs]
            Xs = [torch.zeros((p, s, n), dtype=torch.float64, device="cuda") for n, s, p in shapes]
            st, infos, sts = ctx.batched_solve(ops, [to_dev(C) for C in Cs_h], Xs, restart=20, precision=prec)
            assert st == 0 and all(x == 0 for x in sts)
            assert ctx.tune_entries()[key] == sched          # the forced schedule ran; nothing was tuned
            outs[sched] = ([from_dev(X) for X in Xs], [i.iters for i in infos])
            for op in ops:
                op.close()
            ctx.workspace_check()
        assert len(_lines(cache)) == 2
    ref_X, ref_it = outs[64]
    for sched in (65, 128, 129):
        X, its = outs[sched]
        assert its == ref_it, sched
        for a, b in zip(ref_X, X):
            assert np.array_equal(a, b), sched


def _batched_solve_forced(tmp_path, monkeypatch, tag, shapes, prec, forced, name):
    """One batched solve (FP64 engine: DFMA) with the cache file holding exactly `forced` (key -> value)."""
    import torch
    from paper_2405_09233_gb300 import Context
    probs = [inputs.dense_problem(n, s, p, seed=80 + i) for i, (n, s, p) in enumerate(shapes)]
    cache = tmp_path / name
    cache.write_text("".join(f"{tag} {k} {v}\n" for k, v in forced.items()))
    monkeypatch.setenv("TSTAR_TUNE_CACHE", str(cache))
    with Context(0) as ctx:
        ops = [ctx.op_create_dense(to_dev(pr.A), to_dev(pr.B)) for pr in probs]
        Cs = [to_dev(kr.sylv_apply(pr.A, pr.B, pr.Xstar)) for pr in probs]
        Xs = [torch.zeros((p, s, n), dtype=torch.float64, device="cuda") for n, s, p in shapes]
        st, infos, sts = ctx.batched_solve(ops, Cs, Xs, restart=20, precision=prec)
        assert st == 0 and all(x == 0 for x in sts)
        ent = ctx.tune_entries()
        out = ([from_dev(X) for X in Xs], [i.iters for i in infos], ent)
        for op in ops:
            op.close()
        ctx.workspace_check()
    return out, _lines(cache)


SIMT_SHAPES = [(96, 40, 4), (130, 150, 8), (70, 17, 2), (200, 90, 6)]   # s ragged for 16-, 32- and 64-wide tiles


def _simt_key(esz, shapes):
    return f"bsimt:{esz}:{len(shapes)}" + "".join(f":{n}x{s}x{p // 2 + 1}" for n, s, p in shapes)


@pytest.mark.parametrize("prec", ["fp64", "mixed_fp32"])
def test_batched_cuda_core_tiles_agree_bitwise(tmp_path, monkeypatch, prec):
    """Force each column width of the CUDA-core work-list products (64, 32, 16 columns; FP64 for the DFMA
    residuals and a whole FP64 cycle, FP32 for the inner products of mixed FP32) through the cache file:
    every output entry sums the same products in the same order, so the batched solves agree bit for bit."""
    tag = _device_tag(tmp_path, monkeypatch)
    esz = 8 if prec == "fp64" else 4
    key = _simt_key(esz, SIMT_SHAPES)
    outs = {}
    for bn in (64, 32, 16):
        forced = {key: bn}
        if esz == 4:
            forced[_simt_key(8, SIMT_SHAPES)] = 64              # the FP64 residual products: fixed
        (X, its, ent), lines = _batched_solve_forced(tmp_path, monkeypatch, tag, SIMT_SHAPES, prec, forced,
                                                     f"simt_{prec}_{bn}.txt")
        assert ent[key] == bn                                  # the forced width ran; nothing was tuned
        assert len(lines) == len(forced)
        outs[bn] = (X, its)
    ref_X, ref_it = outs[64]
    for bn in (32, 16):
        X, its = outs[bn]
        assert its == ref_it, bn
        for a, b in zip(ref_X, X):
            assert np.array_equal(a, b), bn


def test_batched_cuda_core_tile_tuned(tmp_path, monkeypatch):
    """Unforced, the FP64 batched solve tunes the CUDA-core column width once and persists it."""
    tag = _device_tag(tmp_path, monkeypatch)
    key = _simt_key(8, SIMT_SHAPES)
    (X, its, ent), lines = _batched_solve_forced(tmp_path, monkeypatch, tag, SIMT_SHAPES, "fp64", {}, "simt_tuned.txt")
    assert ent[key] in (64, 32, 16)
    assert [ln.split()[1:] for ln in lines] == [[key, str(ent[key])]]
