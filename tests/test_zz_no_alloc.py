"""thc_energy_noalloc against thc_energy, through the C ABI (needs a GPU).

The no-alloc entry point serves callers that may not allocate device memory:
a process whose HBM is already held by another runtime's memory pool, or a
loop that must not pay for (or risk) an allocation.  It takes device inputs
and keeps its scratch in a fixed device array.  Two calls in a row with
different inputs must each agree with thc_energy, the second one also
showing that what the first left in the shared scratch does not leak into
its result, and the second call must leave the device's free memory
unchanged.  The first call on a device loads the library's device code for
this entry point (lazy module loading), which commits the fixed array; the
free memory seen around it is printed, not asserted.  This file is collected
last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from synth import make_system, random_amplitudes

pytestmark = pytest.mark.gpu

E_TOL = 1e-9


def test_noalloc_energy_matches_thc_energy_twice():
    torch = pytest.importorskip("torch")
    import __graft_entry__ as g
    g.build()
    import paper_2111_11473_gb300 as pkg
    lib = pkg.load_library()
    o, v, P, G, K = 7, 37, 70, 90, 45
    s = make_system(o, v, P, G, K, seed=11)
    dev = torch.device("cuda:0")
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    Y = torch.from_numpy(s.Y).to(dev)
    Lov = torch.from_numpy(np.ascontiguousarray(s.L[:, :o, o:])).to(dev)
    states = []
    with pkg.Context(s.eps_o, s.eps_v, s.Y, s.L, s.x, s.z, stream=stream) as ctx:
        for seed, t1_scale in ((1, 0.05), (2, 0.0)):
            Zc, t1 = random_amplitudes(P, o, v, seed, t1_scale=t1_scale)
            states.append((torch.from_numpy(Zc).to(dev), torch.from_numpy(t1).to(dev),
                           ctx.energy(Zc, t1)))
    torch.cuda.synchronize(dev)
    free = []
    for k, (Zd, td, E_ref) in enumerate(states):
        e = C.c_double(np.nan)
        before = torch.cuda.mem_get_info(dev)[0]
        st = lib.thc_energy_noalloc(o, v, P, K, Y.data_ptr(), Lov.data_ptr(), Zd.data_ptr(),
                                    td.data_ptr(), C.addressof(e),
                                    C.c_void_p(stream.cuda_stream))
        after = torch.cuda.mem_get_info(dev)[0]
        free.append((before, after))
        assert st == 0, lib.thc_last_error(None).decode()
        print(f"call {k + 1}: |E - thc_energy| = {abs(e.value - E_ref):.2e}, free memory "
              f"{before / 2**20:.1f} -> {after / 2**20:.1f} MiB")
        assert abs(e.value - E_ref) < E_TOL
    # The second call allocates nothing.
    assert free[1][0] == free[1][1]
    # Sizes beyond the fixed scratch are rejected with a reason.
    e = C.c_double(0.0)
    big = 1500
    st = lib.thc_energy_noalloc(o, v, big, K, Y.data_ptr(), Lov.data_ptr(), Y.data_ptr(),
                                Y.data_ptr(), C.addressof(e), None)
    assert st == 1
    assert "exceeds the fixed scratch" in lib.thc_last_error(None).decode()
    # Host inputs are rejected: the kernels read the inputs in place.
    Yh = np.ascontiguousarray(s.Y)
    st = lib.thc_energy_noalloc(o, v, P, K, Yh.ctypes.data, Lov.data_ptr(), Y.data_ptr(),
                                Y.data_ptr(), C.addressof(e), None)
    assert st == 1
    assert "device memory" in lib.thc_last_error(None).decode()
