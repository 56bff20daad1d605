"""GPU parity of batched products (one CUDA graph: parallel sketch branches,
one grouped persistent tensor-core GEMM) through the C ABI."""
import numpy as np
import pytest

import oracle
from helpers import gpu_lib

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    return gpu_lib()


def _problems(rng, count, N=4, e=1, dtype=None):
    """Uneven products: m, l in [1, 600], n in {2048, 4096, 6144}, b = n / 32;
    product p drops block p mod (N + e)."""
    out = []
    for p in range(count):
        m = int(rng.integers(1, 601))
        l = int(rng.integers(1, 601))
        n = int(rng.choice([2048, 4096, 6144]))
        b = n // 32
        mask = ((1 << (N + e)) - 1) & ~(1 << (p % (N + e)))
        A = rng.standard_normal((m, n)).astype(np.float32)
        B = rng.standard_normal((n, l)).astype(np.float32)
        out.append(dict(m=m, n=n, l=l, b=b, N=N, e=e, mask=mask, seed=100 + p, A=A, B=B))
    return out


def _device(ops, probs, in_dtype=torch.float32):
    dev = []
    for q in probs:
        A = torch.from_numpy(q["A"]).cuda().to(in_dtype)
        B = torch.from_numpy(q["B"]).cuda().to(in_dtype)
        C = torch.full((q["m"], q["l"]), float("nan"), dtype=torch.float32, device="cuda")
        plan = ops.plan(q["n"], q["b"], q["N"], q["e"], q["seed"])
        dev.append((A, B, C, plan, q["mask"]))
    return dev


def _bf16_oracle(q, A64=None, B64=None):
    h, s = oracle.hash_tables(q["n"], q["b"], q["N"], q["e"], q["seed"])
    A = q["A"] if A64 is None else A64
    B = q["B"] if B64 is None else B64
    At = oracle.round_bf16(oracle.sketch_left(A, h, s, q["b"]))
    Bt = oracle.round_bf16(oracle.sketch_right(B, h, s, q["b"]))
    return oracle.masked_product(At, Bt, q["b"], q["mask"])


def test_batched_parity_and_replay(ops):
    rng = np.random.default_rng(31)
    probs = _problems(rng, 12)
    dev = _device(ops, probs)
    batch = ops.Batch(dev)
    info = batch.info()
    assert info["count"] == 12 and info["total_tiles"] > 0
    batch.run()
    torch.cuda.synchronize()
    first = [C.clone() for (_, _, C, _, _) in dev]
    for q, (A, B, C, plan, mask) in zip(probs, dev):
        ref = _bf16_oracle(q)
        assert oracle.rel_frob(C.cpu().numpy(), ref) <= 1e-4
        # same sketch kernels and K order as the single-product path
        single = ops.matmul(plan, A, B, mask, "bf16")
        assert oracle.rel_frob(C.cpu().numpy(), single.cpu().numpy().astype(np.float64)) <= 1e-6
    # replays overwrite C with the same bits
    for (_, _, C, _, _) in dev:
        C.fill_(float("nan"))
    batch.run()
    batch.run()
    torch.cuda.synchronize()
    for C0, (_, _, C, _, _) in zip(first, dev):
        assert torch.equal(C0, C)
    assert ops.device_status() == 0
    batch.close()


def test_batched_tuned_and_single_branch(ops):
    rng = np.random.default_rng(32)
    probs = _problems(rng, 9)
    dev = _device(ops, probs)
    ref = [_bf16_oracle(q) for q in probs]
    tuned = ops.Batch(dev, tune=True)
    inf = tuned.info()
    assert inf["tile_n"] in (128, 256) and inf["tuned_ms"] > 0
    tuned.run()
    torch.cuda.synchronize()
    for r, (_, _, C, _, _) in zip(ref, dev):
        assert oracle.rel_frob(C.cpu().numpy(), r) <= 1e-4
    tuned.close()
    # a workspace limit of one packing slot forces one sketch branch
    slot = max(max(ops.sketch_workspace(ops.plan(q["n"], q["b"], q["N"], q["e"], 0), q["m"]),
                   ops.sketch_workspace(ops.plan(q["n"], q["b"], q["N"], q["e"], 0), q["l"])) for q in probs)
    one = ops.Batch(dev, workspace_limit=(slot + 255) // 256 * 256)
    assert one.info()["branches"] == 1
    for (_, _, C, _, _) in dev:
        C.zero_()
    one.run()
    torch.cuda.synchronize()
    for r, (_, _, C, _, _) in zip(ref, dev):
        assert oracle.rel_frob(C.cpu().numpy(), r) <= 1e-4
    one.close()


def test_batched_bf16_inputs(ops):
    rng = np.random.default_rng(33)
    probs = _problems(rng, 5)
    dev = _device(ops, probs, torch.bfloat16)
    batch = ops.Batch(dev)
    batch.run()
    torch.cuda.synchronize()
    for q, (A, B, C, _, _) in zip(probs, dev):
        ref = _bf16_oracle(q, A.float().cpu().numpy().astype(np.float64), B.float().cpu().numpy().astype(np.float64))
        assert oracle.rel_frob(C.cpu().numpy(), ref) <= 1e-4
    batch.close()


def test_batched_argument_errors(ops):
    rng = np.random.default_rng(34)
    probs = _problems(rng, 2)
    dev = _device(ops, probs)
    with pytest.raises(ops.OverSketchError, match="OS_ERR_DTYPE"):
        ops.Batch(dev, gemm_dtype="f32")
    A, B, C, plan, mask = dev[0]
    with pytest.raises(ops.OverSketchError, match="OS_ERR_UNSUPPORTED"):
        ops.Batch([(A, B, C, ops.plan(A.shape[1], 96, 4, 1, 0), mask)])          # b % 64 != 0
    with pytest.raises(ops.OverSketchError, match="OS_ERR_INVALID_ARG"):
        ops.Batch([(A, B, C, ops.plan(A.shape[1] + 64, 64, 4, 1, 0), mask)])     # plan dimension != n
    with pytest.raises(ops.OverSketchError, match="OS_ERR_MASK"):
        ops.Batch([(A, B, C, plan, 1 << 7)])                                     # block past N + e


def test_matmul_batched_device_masks_in_one_captured_graph(ops):
    # oversketch_matmul_batched reads every product's kept blocks from device
    # memory when the work runs: ONE captured graph, replayed with three different
    # straggler sets (including an empty mask: a zero product), matches the oracle
    # every time.  The call allocates nothing (caller workspace), so it can be
    # recorded inside torch's graph capture.
    rng = np.random.default_rng(41)
    probs = _problems(rng, 9)
    probs[3]["m"], probs[3]["A"] = 0, probs[3]["A"][:0]        # an empty product is skipped
    dev = _device(ops, probs)
    plans = [d[3] for d in dev]
    As, Bs, Cs = [d[0] for d in dev], [d[1] for d in dev], [d[2] for d in dev]
    P = probs[0]["N"] + probs[0]["e"]
    masks = torch.zeros(len(probs), dtype=torch.int64, device="cuda")
    ws = torch.empty(ops.matmul_batched_workspace(plans, [A.shape[0] for A in As], [A.shape[1] for A in As],
                                                  [B.shape[1] for B in Bs]), dtype=torch.uint8, device="cuda")
    masks.copy_(torch.tensor([q["mask"] for q in probs], dtype=torch.int64))
    ops.matmul_batched(plans, As, Bs, Cs, masks, workspace=ws)      # first call: library streams, attributes
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ops.matmul_batched(plans, As, Bs, Cs, masks, workspace=ws)
    sets = [[q["mask"] for q in probs],
            [((1 << P) - 1) & ~(0b11 << (p % (P - 1))) for p in range(len(probs))],   # two stragglers each
            [0 if p == 5 else (1 << (p % P)) for p in range(len(probs))]]              # one block / none
    for msk in sets:
        masks.copy_(torch.tensor(msk, dtype=torch.int64))
        for C in Cs:
            C.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for p, (q, C) in enumerate(zip(probs, Cs)):
            if q["m"] == 0:
                continue
            ref = _bf16_oracle(dict(q, mask=msk[p])) if msk[p] else np.zeros((q["m"], q["l"]))
            got = C.cpu().numpy()
            if msk[p]:
                assert oracle.rel_frob(got, ref) <= 1e-4, (p, msk[p])
            else:
                assert np.array_equal(got, ref)
    assert ops.device_status() == 0
