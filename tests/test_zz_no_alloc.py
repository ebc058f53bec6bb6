"""stc_group_keys_static, the grouping entry point that allocates nothing, against the
allocating stc_group_keys on the same keys. It serves callers that cannot allocate device
memory (their memory is already carved up by their own allocator, or allocation is
forbidden after start-up), so its scratch is one fixed device array shared by every call.

This file is collected last on purpose. It passes alone in a fresh process and after the
other tests: the first call on the device sets up the array's address, and several calls
in a row check that each one clears the state the previous call left behind."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stc():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_10094_gb300 import build

    build.build()
    import paper_2410_10094_gb300 as mod

    mod.load()
    return mod


def run_both(stc, keys: np.ndarray, k: int):
    import torch

    kd = torch.from_numpy(keys.view(np.int64)).cuda()
    off_ref, perm_ref = stc.group_keys(kd, k)
    off = torch.full((k + 1,), -1, dtype=torch.int32, device="cuda")
    perm = torch.full((keys.size,), -1, dtype=torch.int32, device="cuda")
    stc.stc_group_keys_static(kd, k, off, perm)
    torch.cuda.synchronize()
    return (off.cpu().numpy(), perm.cpu().numpy().astype(np.int64), off_ref.cpu().numpy(),
            perm_ref.cpu().numpy().astype(np.int64))


def test_static_grouping_matches_allocating_grouping(stc):
    rng = np.random.Generator(np.random.PCG64(20241010))
    big = rng.integers(0, 262_144, 400_000).astype(np.uint64)
    small = rng.integers(0, 1_000, 50_000).astype(np.uint64)
    # Two calls in a row on the same keys, then a smaller key range after a larger one, so a
    # count left over from an earlier call would show.
    for keys, k in [(big, 262_144), (big, 262_144), (small, 1_000), (np.zeros(0, np.uint64), 7)]:
        off, perm, off_ref, perm_ref = run_both(stc, keys, k)
        np.testing.assert_array_equal(off, off_ref)  # offsets: integers, bit-exact
        np.testing.assert_array_equal(np.sort(perm), np.arange(keys.size))
        np.testing.assert_array_equal(keys[perm], keys[perm_ref])  # same key in every slot
        for v in np.unique(keys)[:64]:  # same members in each run (order inside is unspecified)
            a, b = off_ref[v], off_ref[v + 1]
            assert sorted(perm[a:b]) == sorted(perm_ref[a:b])


def test_static_grouping_rejects_oversized_key_range(stc):
    import torch

    keys = torch.zeros(10, dtype=torch.int64, device="cuda")
    off = torch.empty(262_146, dtype=torch.int32, device="cuda")
    perm = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(stc.StcError) as e:
        stc.stc_group_keys_static(keys, 262_145, off, perm)
    assert e.value.status == 1 and "262144" in str(e.value)


def test_static_grouping_allocates_nothing(stc):
    """After one warm-up call, further calls leave the device's free memory and torch's
    allocator untouched: the call's scratch is the fixed array, not an allocation."""
    import torch

    rng = np.random.Generator(np.random.PCG64(20241011))
    keys = torch.from_numpy(rng.integers(0, 100_000, 300_000).astype(np.int64)).cuda()
    off = torch.empty(100_001, dtype=torch.int32, device="cuda")
    perm = torch.empty(keys.numel(), dtype=torch.int32, device="cuda")
    stc.stc_group_keys_static(keys, 100_000, off, perm)  # warm-up: the address look-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(5):
        stc.stc_group_keys_static(keys, 100_000, off, perm)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert torch.cuda.memory_allocated() == alloc0
    assert free1 == free0


def test_static_grouping_wrapper_rejects_bad_arrays(stc):
    """The Python wrapper checks what the C call cannot: sizes, types, layout and device."""
    import torch

    keys = torch.zeros(10, dtype=torch.int64, device="cuda")
    off = torch.empty(8, dtype=torch.int32, device="cuda")
    perm = torch.empty(10, dtype=torch.int32, device="cuda")
    bad = [
        (keys, 7, off[:7], perm),                                   # offsets_out shorter than k + 1
        (keys, 7, off, perm[:9]),                                   # perm_out shorter than n
        (keys, 7, off.to(torch.int64), perm),                       # wrong offsets type
        (keys.to(torch.int32), 7, off, perm),                       # wrong key type
        (keys.cpu(), 7, off, perm),                                 # host keys
        (torch.zeros(20, dtype=torch.int64, device="cuda")[::2], 7, off, perm),  # strided keys
    ]
    for args in bad:
        with pytest.raises(ValueError):
            stc.stc_group_keys_static(*args)
