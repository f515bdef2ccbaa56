"""dem_find_pairs_noalloc: the pair query for callers that cannot allocate device
memory (its scratch is a fixed array inside the library).  Its output must equal
dem_find_pairs's on the same input, on two calls in a row -- the second call also
shows that the shared scratch left by the first call does not leak into the
result.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2301_00611_gb300 as pkg
    return torch, pkg


def _inputs(torch, w, shift_periods=False):
    pos = w.pos
    if shift_periods:
        L = w.cell[0, 0]
        pos = pos + ((workloads.uniform(pos.size, 3).reshape(pos.shape) * 5).astype(int) - 2) * L
    return (torch.tensor(pos, dtype=torch.float64, device="cuda"),
            torch.tensor(w.radius, dtype=torch.float64, device="cuda"))


def _same(a, b):
    # integer outputs: exact equality, rows in the same fixed order
    return all(np.array_equal(x.cpu().numpy(), y.cpu().numpy()) for x, y in zip(a, b))


def test_noalloc_matches_allocating_query_on_two_calls(env):
    torch, pkg = env
    w1 = workloads.periodic_cloud(6000, 21, phi=0.33, inflate=1.05)
    w2 = workloads.box_cloud(4000, 22, phi=0.3, inflate=1.04, wall_mask=0)
    P1, R1 = _inputs(torch, w1, shift_periods=True)
    P2, R2 = _inputs(torch, w2)
    ref1 = pkg.find_pairs(P1, R1, periodic=True, cell=w1.cell, margin=1e-4)
    ref2 = pkg.find_pairs(P2, R2, margin=0.0)
    got1 = pkg.find_pairs(P1, R1, periodic=True, cell=w1.cell, margin=1e-4, noalloc=True)
    got2 = pkg.find_pairs(P2, R2, margin=0.0, noalloc=True)
    assert len(ref1[0]) > 3000 and len(ref2[0]) > 1000
    assert _same(got1, ref1)
    assert _same(got2, ref2)
    again = pkg.find_pairs(P1, R1, periodic=True, cell=w1.cell, margin=1e-4, noalloc=True)
    assert _same(again, ref1)


def test_noalloc_rejects_more_spheres_than_its_scratch_holds(env):
    torch, pkg = env
    n = (1 << 16) + 1
    pos = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    rad = torch.full((n,), 1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DemError) as e:
        pkg.find_pairs(pos, rad, noalloc=True)
    assert e.value.code == 4
    assert "65536" in str(e.value)


def _cudart():
    """The CUDA runtime that torch loaded (by soname), else the toolkit's copy.  The
    default memory pool is a per-device driver object, so any runtime instance in the
    process sees the one that the library's stream-ordered allocations use."""
    import ctypes
    import os
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return ctypes.CDLL(name if os.path.isabs(name) else name)
        except OSError:
            continue
    pytest.skip("no CUDA runtime library found to read the memory-pool counters")


def test_noalloc_call_makes_no_device_allocation(env):
    """The property the entry point exists for.  After a warm-up call, the high-water
    mark of the device's default memory pool (where the allocating query's
    stream-ordered allocations come from) is reset to the memory in use, and the free
    device memory is recorded; a second no-allocation call must move neither.  Control: the allocating
    dem_find_pairs does raise the pool's high-water mark."""
    import ctypes
    torch, pkg = env
    rt = _cudart()
    lib = pkg.load_library()
    dev = torch.cuda.current_device()
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), dev) == 0
    used_cur, used_high = 0x7, 0x8                # cudaMemPoolAttrUsedMem{Current,High}

    def cur():
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, used_cur, ctypes.byref(v)) == 0
        return v.value

    def reset_high():
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, used_high, ctypes.byref(zero)) == 0

    def high():
        v = ctypes.c_uint64(0)
        assert rt.cudaMemPoolGetAttribute(pool, used_high, ctypes.byref(v)) == 0
        return v.value

    def free_bytes():
        f, t = ctypes.c_size_t(), ctypes.c_size_t()
        assert rt.cudaMemGetInfo(ctypes.byref(f), ctypes.byref(t)) == 0
        return f.value

    w = workloads.periodic_cloud(5000, 23, phi=0.33, inflate=1.05)
    P, R = _inputs(torch, w)
    n = w.radius.size
    cap = 8 * n
    I = torch.empty(cap, dtype=torch.int32, device="cuda")
    J = torch.empty(cap, dtype=torch.int32, device="cuda")
    C = torch.empty((cap, 3), dtype=torch.int32, device="cuda")
    H = np.ascontiguousarray(w.cell, dtype=np.float64)
    st = torch.cuda.current_stream().cuda_stream

    def call(fn):
        cnt = ctypes.c_longlong()
        rc = fn(P.data_ptr(), R.data_ptr(), n, 1, H.ctypes.data, 1e-4, cap, I.data_ptr(),
                J.data_ptr(), C.data_ptr(), ctypes.byref(cnt), st)
        assert rc == 0, lib.dem_last_error(None).decode()
        assert 0 < cnt.value <= cap
        return cnt.value

    m0 = call(lib.dem_find_pairs_noalloc)              # warm-up: set-up, module loaded
    torch.cuda.synchronize()
    # other objects of the process (earlier scenes) may hold pool memory: the reset
    # brings the high-water mark down to what is in use now, and the call must not
    # raise it
    reset_high()
    c0 = cur()
    assert high() == c0
    f0 = free_bytes()
    m1 = call(lib.dem_find_pairs_noalloc)
    torch.cuda.synchronize()
    assert m1 == m0
    assert high() == c0
    assert free_bytes() == f0
    # control: the allocating query takes its scratch from that pool
    call(lib.dem_find_pairs)
    torch.cuda.synchronize()
    assert high() > c0
