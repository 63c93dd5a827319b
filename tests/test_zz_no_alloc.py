"""Allocation-free best-move evaluation (tga_eval_best_move_noalloc).

Callers that cannot allocate device memory get the best move of an
instance + solution from a fixed scratch array inside the library.  Its
result must equal the context-based tga_eval_best_move exactly, also when
two calls in a row leave the shared scratch holding another instance's data.
This file is collected last so a failure here never hides another test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2506_17357_gb300 import instances as I  # noqa: E402
from paper_2506_17357_gb300 import tga as T  # noqa: E402


def _noalloc(ls, mask):
    out = torch.zeros(6, dtype=torch.int32, device=ls.device)
    ls.stream.synchronize()
    T.tga_eval_best_move_noalloc(ls.c_inst, ls.c_sol, mask, ls.stream.cuda_stream, out.data_ptr())
    v = out.cpu().numpy()
    return dict(delta=int(v[0]), move_index=int(np.uint32(v[1].view(np.uint32))), op=int(v[2]),
                a=int(v[3]), b=int(v[4]), valid=bool(v[5]))


def test_noalloc_equals_context_path_on_consecutive_calls():
    inst2, sol2 = I.config2(1)                       # VRPTW, 1000 customers
    inst1 = I.cvrp_uniform(300, 7)
    sol1 = I.random_split_solution(inst1, 8)
    inst3 = I.vrpspdtw(500, 9)                       # with pickups
    sol3 = I.random_split_solution(inst3, 10)
    cases = [(inst2, sol2, I.MASK_CONFIG2), (inst1, sol1, I.MASK_CVRP_MIXED), (inst3, sol3, I.MASK_ALL),
             (inst2, sol2, I.MASK_EXT)]                # with the swaps of runs
    for inst, sol, mask in cases:                    # two calls in a row, different data
        ls = T.LocalSearch(inst, sol, mask).build()
        try:
            ref = ls.eval_best_move()
            got = _noalloc(ls, mask)
            assert got == ref
            # move the context one step on and compare again
            ls.apply_current_move()
            ref2 = ls.eval_best_move()
            got2 = _noalloc(ls, mask)
            assert got2 == ref2 and got2 != got
        finally:
            ls.close()


def test_noalloc_allocates_nothing_on_a_warm_call():
    """The entry point's defining property: once its first call on the device
    has looked up the scratch address, a call changes neither the device's
    free memory nor torch's reserved memory (no cudaMalloc, no stream-ordered
    pool growth, no allocation through torch)."""
    inst, sol = I.config2(1)
    ls = T.LocalSearch(inst, sol, I.MASK_CONFIG2).build()
    try:
        first = _noalloc(ls, I.MASK_CONFIG2)                 # warm: scratch address looked up
        out = torch.zeros(6, dtype=torch.int32, device=ls.device)
        torch.cuda.synchronize()
        free0, reserved0 = torch.cuda.mem_get_info(ls.device)[0], torch.cuda.memory_reserved(ls.device)
        for _ in range(3):
            T.tga_eval_best_move_noalloc(ls.c_inst, ls.c_sol, I.MASK_CONFIG2, ls.stream.cuda_stream,
                                         out.data_ptr())
        torch.cuda.synchronize()
        free1, reserved1 = torch.cuda.mem_get_info(ls.device)[0], torch.cuda.memory_reserved(ls.device)
        assert (free1, reserved1) == (free0, reserved0)
        v = out.cpu().numpy()
        assert (int(v[0]), int(v[2]), int(v[3]), int(v[4])) == (first["delta"], first["op"], first["a"], first["b"])
    finally:
        ls.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    inst = I.cvrp_uniform(1300, 3)                   # n + m + 1 > 1280
    sol = I.random_split_solution(inst, 4)
    ls = T.LocalSearch(inst, sol, I.MASK_CONFIG1)
    try:
        out = torch.zeros(6, dtype=torch.int32, device=ls.device)
        with pytest.raises(T.TGAError) as e:
            T.tga_eval_best_move_noalloc(ls.c_inst, ls.c_sol, I.MASK_CONFIG1, ls.stream.cuda_stream,
                                         out.data_ptr())
        assert e.value.code == T.TGA_ERR_RANGE
    finally:
        ls.close()
