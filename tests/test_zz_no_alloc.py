"""The allocation-free entry point, mcmcmc_run_noalloc, against mcmcmc_run.

Some callers of this library cannot allocate device memory: applications
whose GPU memory is owned by their own pool allocator, latency-critical loops
that cannot pay for cudaMalloc's implicit synchronisation, plug-in hosts that
forbid libraries from allocating.  mcmcmc_run_noalloc serves them from a fixed
device array; these checks run it twice in a row on different problems (the
array keeps the previous call's contents) and compare each result with the
ordinary entry point's on the same inputs: bit-exact spins and energies for
+-J couplings, and for Gaussian couplings the parity tolerance of the other
GPU tests (energy per spin within 1e-5).

This file is named to be collected last.
"""
import numpy as np
import pytest

from paper_2102_05613_gb300 import inputs, sk

from gpu_util import need_gpu

pytestmark = pytest.mark.gpu

E_PER_SPIN_TOL = 1e-5


def _with_allocating_api(J, init, *, K, rule, beta, seed, stream_id, steps, scale):
    inst = sk.Instance(J, scale=scale)
    run = sk.Run(inst, chains=init.shape[0], K=K, rule=rule, beta=beta, seed=seed,
                 stream_id=stream_id, init=init)
    run.advance(steps)
    spins, _ = run.state()
    E = inst.energy(spins)
    run.close()
    inst.close()
    return spins, E


CASES = [
    # N, kind, chains, K, rule, beta, scale, steps
    (100, sk.SK_J_PM1, 6, 33, sk.SK_RULE_MCMCMC, 0.7, 1.0, 700),
    (200, sk.SK_J_GAUSS, 8, 128, sk.SK_RULE_MCMCMC, 1.0, 1.0, 500),
    (64, sk.SK_J_PM1, 4, 1, sk.SK_RULE_METROPOLIS, 1.0, 0.125, 900),
]


@pytest.mark.parametrize("order", [(0, 1), (1, 2), (2, 0)])
def test_noalloc_matches_allocating_run_on_two_calls_in_a_row(order):
    torch = need_gpu()
    for idx in order:
        N, kind, chains, K, rule, beta, scale, steps = CASES[idx]
        J = inputs.couplings(N, kind, 300 + idx)
        init = inputs.initial_spins(chains, N, 400 + idx)
        Jd = torch.from_numpy(J).cuda()
        Sd = torch.from_numpy(init).cuda()
        Ed = torch.full((chains,), float("nan"), dtype=torch.float64, device="cuda")
        sk.run_noalloc(Jd, Sd, Ed, scale=scale, K=K, rule=rule, beta=beta, seed=11 + idx,
                       stream_id=idx, steps=steps)
        torch.cuda.synchronize()
        spins = Sd.cpu().numpy()
        E = Ed.cpu().numpy()
        ref_spins, ref_E = _with_allocating_api(J, init, K=K, rule=rule, beta=beta, seed=11 + idx,
                                                stream_id=idx, steps=steps, scale=scale)
        if kind == sk.SK_J_PM1:
            assert np.array_equal(spins, ref_spins)
            assert np.array_equal(E, ref_E)
        else:
            assert np.array_equal(spins, ref_spins)
            assert np.abs(E - ref_E).max() / N <= E_PER_SPIN_TOL


def test_noalloc_rejects_problems_beyond_its_array():
    torch = need_gpu()
    N, chains = 2048, 1024          # 16 MiB of couplings alone
    Jd = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    Sd = torch.ones((chains, N), dtype=torch.int8, device="cuda")
    Ed = torch.zeros((chains,), dtype=torch.float64, device="cuda")
    with pytest.raises(sk.SKError) as e:
        sk.run_noalloc(Jd, Sd, Ed, K=8, steps=10)
    assert e.value.status == sk.SK_ERR_INVALID_ARG
    assert "allocation-free limit" in str(e.value)
