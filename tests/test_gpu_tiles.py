"""Far-field pair tiles and their autotuner: every tile variant produces the same V
bit for bit (each entry is computed by one thread with the same operations), and the
autotuned choice is timed once per context, precision and size class."""
import numpy as np
import pytest

from paper_1901_08393_gb300 import bem, inputs

pytestmark = pytest.mark.gpu


def _ctx():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    return bem.Context()


@pytest.mark.parametrize("prec", [bem.PREC_F64, bem.PREC_F32, bem.PREC_DF64], ids=["f64", "f32", "df64"])
@pytest.mark.parametrize("m", [inputs.workload_polycube_adaptive(), inputs.cube_mesh(13)], ids=lambda m: m.name)
def test_every_tile_variant_gives_the_same_operator(m, prec):
    ctx = _ctx()
    mesh = bem.Mesh.upload(ctx, m.verts, m.tris)
    ref = bem.Operator.assemble(mesh, precision=prec, tile=1).read()
    for v in range(2, bem.FAR_TILE_VARIANTS + 1):
        assert np.array_equal(bem.Operator.assemble(mesh, precision=prec, tile=v).read(), ref), v
    assert np.array_equal(bem.Operator.assemble(mesh, precision=prec, tile=0).read(), ref)
    # incremental reassembly with another variant: the same as the full assembly
    rng = np.random.default_rng(2)
    fine = bem.refine(mesh, (rng.random(m.N) < 0.2).astype(np.uint8))
    coarse = bem.Operator.assemble(mesh, precision=prec, tile=4)
    inc = bem.Operator.update(fine, coarse)
    assert np.array_equal(inc.read(), bem.Operator.assemble(fine, precision=prec, tile=2).read())
    ctx.close()


def test_autotune_is_timed_once_per_size_class():
    ctx = _ctx()
    assert ctx.far_tiles() == [[0] * 4] * 3
    small = bem.Mesh.upload(ctx, *[getattr(inputs.workload_polycube_adaptive(), k) for k in ("verts", "tris")])
    bem.Operator.assemble(small, precision=bem.PREC_DF64)
    tiles = ctx.far_tiles()
    assert 1 <= tiles[bem.PREC_DF64][0] <= bem.FAR_TILE_VARIANTS
    assert tiles[bem.PREC_DF64][1:] == [0, 0, 0] and tiles[bem.PREC_F64] == [0] * 4
    # a second assembly of the class launches no timing runs: as many kernels as a fixed tile
    n0 = ctx.launch_count()
    bem.Operator.assemble(small, precision=bem.PREC_DF64)
    n_auto = ctx.launch_count() - n0
    n0 = ctx.launch_count()
    bem.Operator.assemble(small, precision=bem.PREC_DF64, tile=3)
    assert ctx.launch_count() - n0 == n_auto
    assert ctx.far_tiles() == tiles
    # another size class is timed on its own
    big = bem.Mesh.upload(ctx, inputs.cube_mesh(13).verts, inputs.cube_mesh(13).tris)  # 2,028 triangles
    bem.Operator.assemble(big, precision=bem.PREC_DF64)
    assert 1 <= ctx.far_tiles()[bem.PREC_DF64][1] <= bem.FAR_TILE_VARIANTS
    with pytest.raises(bem.BemError) as e:
        bem.Operator.assemble(small, tile=bem.FAR_TILE_VARIANTS + 1)
    assert e.value.code == bem.BEM_ERR_INVALID
    ctx.close()


def test_batch_times_its_size_classes_before_any_graph():
    ctx = _ctx()
    ms = [inputs.cube_mesh(k) for k in (3, 6, 14)]  # 108, 432 and 2,352 triangles
    meshes = [bem.Mesh.upload(ctx, m.verts, m.tris) for m in ms]
    bt = bem.Batch(ctx, meshes, precision=bem.PREC_DF64, use_graph=True)
    tiles = ctx.far_tiles()[bem.PREC_DF64]
    assert tiles[0] >= 1 and tiles[1] >= 1
    r1 = bt.run()
    r2 = bt.run()  # graph replay
    assert [r["cap"] for r in r1] == [r["cap"] for r in r2]
    for m, mesh, r in zip(ms, meshes, r1):
        cap, _, _ = bem.solve_capacity(bem.Operator.assemble(mesh, precision=bem.PREC_DF64, tile=1), tol=1e-10)
        assert abs(r["cap"] / cap - 1) < 1e-9
    ctx.close()
