"""The depth sort of the tile lists (the "depth ordered list" of Eq. 2), bit for bit against numpy's
sort of the same 64-bit keys ((float32 depth bits << 32) | Gaussian index, ascending: depth order
with equal depths in index order). List lengths cover every path of the library's sort: the
warp-per-list radix sort (up to 1024 keys), the CTA radix sort of the queued lists (1025..4096)
and sorted runs plus merge-path merges beyond; depth distributions cover narrow and wide ranges,
ranges across powers of two, many equal depths and a list of one depth."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda"

LENGTHS = [0, 1, 2, 3, 31, 32, 33, 255, 256, 257, 700, 1023, 1024, 1025, 1500, 2048, 2049, 3000, 4095, 4096,
           4097, 9000, 20000]


@pytest.fixture(scope="module")
def icgs():
    from paper_2604_17155_gb300 import build as B
    B.build()
    from paper_2604_17155_gb300 import icgs as I
    I.load()
    return I


def _depths(rng, kind, n):
    if kind == "uniform":
        d = rng.uniform(2.0, 6.0, n)
    elif kind == "octaves":  # across 0.5, 1, 2 (the depth word's exponent changes)
        d = rng.uniform(0.4, 3.0, n)
    elif kind == "wide":
        d = np.exp(rng.uniform(np.log(1e-3), np.log(1e3), n))
    elif kind == "narrow":
        d = 5.0 + rng.uniform(0.0, 1e-4, n)
    elif kind == "few":  # five depths: long runs of equal depth
        d = rng.choice(np.array([0.7, 1.0, 1.3, 2.5, 9.0]), n)
    else:  # "one": every key of the list at one depth
        d = np.full(n, 3.0)
    return d.astype(np.float32)


def _lists(seed, lengths, kinds):
    rng = np.random.default_rng(seed)
    keys, off = [], [0]
    for i, n in enumerate(lengths):
        kind = kinds[i % len(kinds)]
        depth_bits = _depths(rng, kind, n).view(np.uint32).astype(np.uint64)
        idx = rng.choice(3_000_000, size=n, replace=False).astype(np.uint64)
        k = (depth_bits << np.uint64(32)) | idx
        if kind != "one" and n > 8:  # plant equal depths with other indices
            j = rng.integers(1, n, n // 8)
            k[j] = (k[j - 1] & np.uint64(0xFFFFFFFF00000000)) | (k[j] & np.uint64(0xFFFFFFFF))
        keys.append(k)
        off.append(off[-1] + n)
    return np.concatenate(keys).view(np.int64), np.array(off, np.int64)


def _expected(keys, off):
    out = keys.copy()
    for t in range(len(off) - 1):
        b, e = off[t], off[t + 1]
        out[b:e] = np.sort(keys[b:e])
    return out


KINDS = ["uniform", "octaves", "wide", "narrow", "few", "one"]


def test_sort_every_path_bit_exact(icgs):
    lengths = [n for n in LENGTHS for _ in range(len(KINDS))]
    keys, off = _lists(7, lengths, KINDS)
    assert all(len(np.unique(keys[off[t]:off[t + 1]])) == off[t + 1] - off[t] for t in range(len(off) - 1))
    g_keys = torch.tensor(keys, device=DEV)
    icgs.sort_tile_lists(torch.tensor(off, dtype=torch.int32, device=DEV), g_keys)
    got = g_keys.cpu().numpy()
    exp = _expected(keys, off)
    bad = np.nonzero(got != exp)[0]
    assert bad.size == 0, f"{bad.size} keys out of place, first at {bad[:5]}"


def test_sort_many_lists_headline_lengths(icgs):
    """Thousands of lists with the length mix of a large scene (mean about 850 keys, a tail past
    4096), so that many warps and CTAs of the persistent kernels run at once."""
    rng = np.random.default_rng(11)
    lengths = np.minimum(rng.exponential(850.0, 3000).astype(np.int64), 12000)
    keys, off = _lists(12, lengths, KINDS[:5])
    g_keys = torch.tensor(keys, device=DEV)
    icgs.sort_tile_lists(torch.tensor(off, dtype=torch.int32, device=DEV), g_keys)
    assert np.array_equal(g_keys.cpu().numpy(), _expected(keys, off))


def test_sort_cut_at_key_count(icgs):
    """Keys past nkeys are left alone; the list that crosses nkeys is sorted up to it."""
    keys, off = _lists(13, [500, 1500, 3000], ["uniform"])
    cut = 500 + 1500 + 1000
    buf = torch.tensor(keys, device=DEV)
    icgs.sort_tile_lists(torch.tensor(off, dtype=torch.int32, device=DEV), buf[:cut])
    got = buf.cpu().numpy()
    exp = _expected(keys[:cut], np.minimum(off, cut))
    assert np.array_equal(got[:cut], exp)
    assert np.array_equal(got[cut:], keys[cut:])


def test_sort_rejects_small_workspace(icgs):
    import ctypes
    lib = icgs.load()
    off = torch.zeros(3, dtype=torch.int32, device=DEV)
    keys = torch.zeros(4, dtype=torch.int64, device=DEV)
    need = lib.icgs_sort_workspace_size(2, 4)
    ws = torch.empty(need, dtype=torch.uint8, device=DEV)
    st = lib.icgs_sort_tile_lists(ctypes.c_void_p(off.data_ptr()), ctypes.c_void_p(keys.data_ptr()), 2, 4,
                                  ctypes.c_void_p(ws.data_ptr()), need - 1, None)
    assert st == icgs.ERR_WORKSPACE_TOO_SMALL
