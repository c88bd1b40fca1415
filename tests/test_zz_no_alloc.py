"""ngb_deliver_spikes_noalloc: the delivery entry point for callers that
cannot allocate device memory.  Through the C ABI, with every device buffer
owned by the caller (here PyTorch), its ring-buffer contents must equal what
ngb_simulate's own delivery left pending, call after call.

The network is simulated with the regular API; the test then replays the
last max-delay steps' recorded spikes through the allocation-free entry point,
one call per step (zeroing each slot as the update would consume it), and
compares every pending slot with ngb_get_input: exactly in fixed-point mode,
within 1e-5 of the summed weight magnitudes in FP32 mode.  This file is
collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2007_14236_gb300 import workloads as W

pytestmark = pytest.mark.gpu


class CsrDevice(C.Structure):
    _fields_ = [("src_syn", C.c_void_p), ("src_grp", C.c_void_p), ("grp_start", C.c_void_p),
                ("grp_delay", C.c_void_p), ("tgt", C.c_void_p), ("weight", C.c_void_p),
                ("num_neurons", C.c_int64), ("num_synapses", C.c_int64), ("num_groups", C.c_int64),
                ("weight_dtype", C.c_int32), ("pad_", C.c_int32)]


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_14236_gb300 import ngb
    L = ngb.load()
    L.ngb_deliver_spikes_noalloc.argtypes = [C.POINTER(CsrDevice), C.c_void_p, C.c_int64, C.c_void_p, C.c_int64,
                                             C.c_int32, C.c_int32, C.c_int64, C.c_void_p]
    L.ngb_deliver_spikes_noalloc.restype = C.c_int
    return torch, ngb, L


def _device_csr(torch, sim, keep):
    """The handle's CSR copied into caller-owned device tensors (group tables
    rebuilt from the per-synapse delays)."""
    st = sim.stats()
    N = st["num_neurons"]
    sp = sim.src_ptr().astype(np.int64)
    syn = sim.synapses()
    K = len(syn["tgt"])
    src = np.repeat(np.arange(N), np.diff(sp))
    d = syn["delay"].astype(np.int64)
    new = np.ones(K, dtype=bool)
    new[1:] = (src[1:] != src[:-1]) | (d[1:] != d[:-1])
    starts = np.flatnonzero(new)
    grp_start = np.append(starts, K).astype(np.int64)
    grp_delay = d[starts].astype(np.int16)
    src_grp = np.searchsorted(starts, sp).astype(np.int32)  # first group at or after each row start
    tw = (syn["tgt"].astype(np.uint64) | (syn["receptor"].astype(np.uint64) << 30)).astype(np.uint32)
    dev = dict(src_syn=torch.from_numpy(sp).cuda(), src_grp=torch.from_numpy(src_grp).cuda(),
               grp_start=torch.from_numpy(grp_start).cuda(), grp_delay=torch.from_numpy(grp_delay).cuda(),
               tgt=torch.from_numpy(tw.view(np.int32)).cuda(), w=torch.from_numpy(syn["weight"]).cuda())
    keep.append(dev)
    csr = CsrDevice(dev["src_syn"].data_ptr(), dev["src_grp"].data_ptr(), dev["grp_start"].data_ptr(),
                    dev["grp_delay"].data_ptr(), dev["tgt"].data_ptr(), dev["w"].data_ptr(), N, K,
                    len(starts), 0, 0)
    return csr, syn


def _replay_and_compare(env, fixed):
    torch, ngb, L = env
    spec = W.balanced_lif(n=1000, indegree=100, seed=3, V_init_sd=5.0)
    spec.conns[0].delay = W.Dist("normal", 1.5, 0.75)  # several delay groups per source
    sim = ngb.from_spec(spec, deterministic=fixed)
    sim.simulate(600)
    st = sim.stats()
    N, Ls, D, T = st["num_neurons"], st["ring_slots"], st["max_delay_steps"], st["steps"]
    keep = []
    csr, syn = _device_csr(torch, sim, keep)
    ring = torch.zeros((Ls, 1, N), dtype=torch.int64 if fixed else torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ids, steps = sim.spikes(t0=T - D, t1=T)
    calls = 0
    for s in range(T - D, T):
        ring[s & (Ls - 1)].zero_()  # the update of step s consumes its slot
        sp = torch.from_numpy(ids[steps == s].astype(np.int32)).cuda()
        rc = L.ngb_deliver_spikes_noalloc(C.byref(csr), C.c_void_p(sp.data_ptr() if len(sp) else None), len(sp),
                                          C.c_void_p(ring.data_ptr()), Ls, 1, int(fixed), s, C.c_void_p(stream))
        assert rc == 0, L.ngb_last_error(None)
        calls += 1
    torch.cuda.synchronize()
    assert calls >= 2 and len(ids) > 20
    got = ring.cpu().numpy()
    # summed weight magnitudes pending per slot and target (the FP32 tolerance scale)
    sp = sim.src_ptr().astype(np.int64)
    absw = np.zeros((D + 1, N))
    for sid, sstep in zip(ids, steps):
        j = np.arange(sp[sid], sp[sid + 1])
        arrive = sstep + syn["delay"][j].astype(np.int64)
        ok = arrive >= T
        np.add.at(absw, (arrive[ok] - T, syn["tgt"][j][ok].astype(np.int64)), np.abs(syn["weight"][j][ok]))
    for off in range(D + 1):
        ref = sim.input(0, off)
        mine = got[(T + off) & (Ls - 1), 0]
        if fixed:
            assert np.array_equal((mine.astype(np.float64) * 2.0**-32).astype(np.float32), ref), off
        else:
            assert np.all(np.abs(mine.astype(np.float64) - ref) <= 1e-5 * absw[off] + 1e-6), off
    sim.close()


def test_noalloc_matches_simulate_fixed_point(env):
    _replay_and_compare(env, fixed=True)
    _replay_and_compare(env, fixed=True)  # the static scratch keeps the last call's contents


def test_noalloc_matches_simulate_fp32(env):
    _replay_and_compare(env, fixed=False)


def test_noalloc_rejects_too_many_spikes(env):
    torch, ngb, L = env
    csr = CsrDevice(1, 1, 1, 1, 1, 1, 10, 0, 0, 0, 0)  # never dereferenced: the size check comes first
    rc = L.ngb_deliver_spikes_noalloc(C.byref(csr), C.c_void_p(1), 4097, C.c_void_p(1), 16, 1, 0, 0, None)
    assert rc == -1 and b"n_spikes" in L.ngb_last_error(None)
