"""Failure paths, made on the host or with short device limits -- no test
here faults, traps or hangs the GPU.

* Bounded device walks that run out report SW_ERR_TIMEOUT: the global
  union-find walk cap of a sweep (sw_params.walk_cap), the round cap of the
  label-equivalence labeller (max_iter) and the idle-poll limit of the Wolff
  growth (sw_wolff_set_wait_limit).  The handle then refuses further work,
  and a fresh handle on the same device still computes bit-exact results.
* An allocator that fails (installed through sw_set_allocator, failing
  after k successful blocks) makes every creating call return SW_ERR_NOMEM
  and give back every block it took."""

import numpy as np
import pytest

import oracle
import paper_1208_2080_gb300 as sw
import synth

pytestmark = pytest.mark.gpu


def _code(excinfo):
    return excinfo.value.code


def test_sweep_walk_cap_reports_timeout_and_the_handle_stays_failed():
    # an all-zero start at 0.9 T_c: one cluster spans every tile, so the
    # merge walks through the global union-find are longer than one step
    L, q, T = 1024, 2, 0.9 * sw.tc(2)
    with sw.Sim(L, q, T, 3, init="zero", walk_cap=1) as s:
        s.sweep(3)
        with pytest.raises(sw.SwError) as e:
            s.sync()
        assert _code(e) == sw._binding.SW_ERR_TIMEOUT
        with pytest.raises(sw.SwError) as e:
            s.sweep(1)
        assert _code(e) == sw._binding.SW_ERR_TIMEOUT
        with pytest.raises(sw.SwError) as e:
            s.measure()
        assert _code(e) == sw._binding.SW_ERR_TIMEOUT
    # the context is still usable: a fresh handle is bit-exact
    with sw.Sim(64, 3, sw.tc(3), 5) as s:
        s.sweep(4)
        got = s.spins()
    assert np.array_equal(got, oracle.run(64, 3, sw.tc(3), 5, 4)[0])


def test_generous_walk_cap_changes_nothing():
    L, q, T, seed = 200, 2, sw.tc(2), 8
    with sw.Sim(L, q, T, seed, walk_cap=1 << 20) as s:
        s.sweep(5)
        got = s.spins()
    assert np.array_equal(got, oracle.run(L, q, T, seed, 5)[0])


def test_label_equivalence_round_cap_reports_timeout():
    import torch
    L = 256
    b = synth.random_bonds(L, 0.5, 21)
    packed = torch.from_numpy(sw.pack_bonds(b).reshape(-1).copy()).cuda()
    roots = torch.empty(L * L, dtype=torch.int32, device="cuda")
    rounds = sw.label_bonds_le(L, packed, roots)
    assert rounds > 2
    with pytest.raises(sw.SwError) as e:
        sw.label_bonds_le(L, packed, roots, max_iter=1)
    assert _code(e) == sw._binding.SW_ERR_TIMEOUT
    # the same call with enough rounds still labels correctly
    sw.label_bonds_le(L, packed, roots, max_iter=rounds)
    torch.cuda.synchronize()
    assert np.array_equal(roots.cpu().numpy().view(np.uint32).reshape(L, L), oracle.label(b))


def test_wolff_growth_wait_limit_reports_timeout():
    # an ordered start at T_c / 2: the clusters cover most of the lattice, and
    # with one idle poll allowed the growth warps that find the queue empty
    # for a moment give up
    L, q = 256, 2
    with sw.Wolff(L, q, 0.5 * sw.tc(q), 4, init="zero", mode="grow") as w:
        w.set_wait_limit(1)
        w.step(3)
        with pytest.raises(sw.SwError) as e:
            w.sync()
        assert _code(e) == sw._binding.SW_ERR_TIMEOUT
        with pytest.raises(sw.SwError):
            w.step(1)
    with sw.Wolff(64, 3, sw.tc(3), 6, mode="grow") as w:
        w.set_wait_limit(0)  # the default again
        w.step(10)
        got = w.spins()
        w.sync()
    assert np.array_equal(got, oracle.wolff_run(64, 3, sw.tc(3), 6, 10,
                                                spins=oracle.init_spins(64, 3, 6))[0])


class _FailingAllocator:
    """Device blocks from PyTorch's caching allocator until `ok` blocks have
    been handed out (None: no limit), NULL after that; counts what is taken
    and given back."""

    def __init__(self, ok=None):
        import torch
        self.ok, self.taken, self.live = ok, 0, {}

        def alloc(nbytes, _ctx):
            if self.ok is not None and self.taken >= self.ok:
                return None
            self.taken += 1
            p = int(torch.cuda.caching_allocator_alloc(int(nbytes)))
            self.live[p] = int(nbytes)
            return p

        def free(ptr, nbytes, _ctx):
            assert self.live.pop(int(ptr)) == int(nbytes)
            torch.cuda.caching_allocator_delete(int(ptr))

        self.fns = (sw._binding.ALLOC_FN(alloc), sw._binding.FREE_FN(free))

    def __enter__(self):
        sw._binding.check(sw.lib().sw_set_allocator(self.fns[0], self.fns[1], None), "sw_set_allocator")
        return self

    def __exit__(self, *a):
        sw._binding.use_torch_allocator()


def _creators():
    import torch
    L = 300
    packed = torch.from_numpy(sw.pack_bonds(synth.random_bonds(L, 0.5, 3)).reshape(-1).copy()).cuda()
    roots = torch.empty(L * L, dtype=torch.int32, device="cuda")

    def label():
        sw.label_bonds(L, packed, roots, label_bits=32)
        return None

    return {
        "lattice": lambda: sw.Sim(512, 3, 1.0, 1),
        "replica batch": lambda: sw.Batch([64, 128], [2, 3], [1.0, 1.1], [1, 2]),
        "Wolff (labelling buffers taken at creation)": lambda: sw.Wolff(128, 2, 1.0, 1),
        "labelling of given bonds (per-call scratch)": label,
    }


def test_failing_allocator_gives_nomem_and_leaks_nothing():
    for name, make in _creators().items():
        # how many blocks the call takes when nothing fails
        with _FailingAllocator() as a:
            h = make()
            need = a.taken
            if h is not None:
                h.close()
        assert need > 0 and not a.live, name
        # failing at every block in turn: SW_ERR_NOMEM, every block given back
        for ok in range(need):
            with _FailingAllocator(ok) as a:
                with pytest.raises(sw.SwError) as e:
                    make()
                assert _code(e) == sw._binding.SW_ERR_NOMEM, (name, ok)
            assert not a.live, (name, ok, len(a.live))
    # with the usual allocator again, a lattice is bit-exact
    with sw.Sim(64, 3, sw.tc(3), 5) as s:
        s.sweep(2)
        assert np.array_equal(s.spins(), oracle.run(64, 3, sw.tc(3), 5, 2)[0])
