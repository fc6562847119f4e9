"""Full-size RowSel checks that cover EVERY output, at the 32-client workload
(N=4096, 2 limbs, 256x64 DB) and the large-DB workload (N=4096, 2 limbs,
1024x128 DB = 4 GiB, 128 clients), in the launch configurations the bench
times (tensor-core tile variants and the CUDA-core path).

Three checks, each with an answer fixed by the mathematics rather than by
the GPU:
  - the oracle (plain definition, Sec. 2.3 GEMM) on one slot in each of 64
    eight-slot groups spread over the whole (limb, slot) range, at a varying
    position inside the group;
  - linearity of the per-slot GEMM (Sec. 2.3): RowSel(ct1) + RowSel(ct2) equals
    RowSel(ct1 + ct2 mod q) element by element over all B*D1*2*L*N outputs,
    with uniform full-range residues;
  - one-hot selection (Sec. 2.2): toy noiseless RLWE queries
    ct_i = (a_i, a_i (.) s + [i == i*_c]) with a distinct i*_c per client;
    every output decrypts, b - a (.) s, to DB[i*_c][j] exactly.
Exact integer work: tolerance 0.
"""

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

# (path, tile variant): the tensor-core fused kernel with and without the
# ingest lookahead, its SM-pair form, the tensor-memory kernel (12 digit
# products) and its SM-pair form, and the CUDA-core path's default tiles.
RUNS = [(4, 0), (4, 3), (4, 7), (4, 8), (4, 9), (1, None)]


@pytest.fixture(scope="module")
def g():
    from tests import gpu_util
    return gpu_util.lib()


class FullSize:
    """One full-size workload on the device: DB (p-major copy kept for the
    checks), uniform ciphertexts ct1, ct2, ct3 = ct1 + ct2 mod q, and a toy
    RLWE query batch."""

    def __init__(self, g, name):
        import torch
        cfg = synth.config_shapes(name)
        self.g, self.name = g, name
        self.N, self.L, self.D0, self.D1 = cfg["N"], cfg["L"], cfg["D0"], cfg["D1"]
        self.B = cfg["B"] if isinstance(cfg["B"], int) else max(cfg["B"])
        self.seed, self.primes = cfg["seed"], list(cfg["primes"])
        N, L, D0, D1, B = self.N, self.L, self.D0, self.D1, self.B
        self.params = g.gpir_params_create(N, self.primes)
        self.db = torch.empty((D0, D1, L, N), dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(self.db, self.db.numel(), 0, self.seed, synth.TAG_DB, self.params, N)
        self.h = g.gpir_db_upload(self.params, D0, D1, self.db, True, 0)
        self.q32 = torch.tensor(self.primes, dtype=torch.int32, device="cuda").view(1, L, 1)
        self.ct1 = torch.empty((B, D0, 2, L, N), dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(self.ct1, self.ct1.numel(), 0, self.seed, synth.TAG_CT, self.params, N)
        self.ct2 = torch.empty_like(self.ct1)
        g.gpir_fill_uniform(self.ct2, self.ct2.numel(), 0, self.seed + 77, synth.TAG_CT, self.params, N)
        self.ct3 = torch.empty_like(self.ct1)
        for c in range(B):       # per client: bounded temporaries
            s = self.ct1[c] + self.ct2[c]                       # < 2^29: no int32 overflow
            self.ct3[c] = s - self.q32 * (s >= self.q32).to(torch.int32)
        # toy RLWE one-hot batch: client c selects row i*_c, secret s_c
        self.istar = [(c * 37 + 5) % D0 for c in range(B)]
        self.sec = torch.empty((B, L, N), dtype=torch.int32, device="cuda")
        g.gpir_fill_uniform(self.sec, self.sec.numel(), 0, self.seed, synth.TAG_SECRET, self.params, N)
        self.ctq = torch.empty_like(self.ct1)
        tmp = torch.empty((D0, L, N), dtype=torch.int32, device="cuda")
        q64 = self.q32.long()
        for c in range(B):
            g.gpir_fill_uniform(tmp, tmp.numel(), 0, self.seed * 1000 + c, synth.TAG_MASK, self.params, N)
            self.ctq[c, :, 0] = tmp
            b = (tmp.long() * self.sec[c].long().unsqueeze(0)) % q64
            b[self.istar[c]] = (b[self.istar[c]] + 1) % q64[0]
            self.ctq[c, :, 1] = b.to(torch.int32)
        del tmp
        torch.cuda.synchronize()

    def run(self, ct, path, variant):
        import torch
        out = torch.full((self.B, self.D1, 2, self.L, self.N), -1, dtype=torch.int32, device="cuda")
        if variant is not None:
            self.g.gpir_set_variant(self.h, self.B, path, variant)
        self.g.gpir_rowsel_batch(self.h, self.B, ct, out, path)
        torch.cuda.synchronize()
        self.g.gpir_sync(None, 60000)
        return out

    def spread_slots(self, n_groups=64):
        groups = self.L * self.N // 8
        out = []
        for k in range(n_groups):
            grp = (k * groups) // n_groups
            t = grp * 8 + (k * 3) % 8
            out.append((t // self.N, t % self.N))
        return out

    def close(self):
        self.g.gpir_db_free(self.h)
        self.g.gpir_params_destroy(self.params)


@pytest.fixture(scope="module", params=["c2_rowsel", "c4_large"])
def work(request, g):
    import torch
    w = FullSize(g, request.param)
    # oracle on 64 spread slots of the first ciphertext batch (host-generated,
    # same counter-based streams as the device fill)
    slots = w.spread_slots()
    ct_s = synth.ct_slots(w.seed, w.B, w.D0, w.L, w.N, w.primes, slots)      # [B][D0][2][S]
    db_s = synth.db_slots(w.seed, w.D0, w.D1, w.L, w.N, w.primes, slots)     # [D0][D1][S]
    w.slots = slots
    w.want = [oracle.rowsel(ct_s[:, :, :, None, k:k + 1], db_s[:, :, None, k:k + 1], [w.primes[l]])[..., 0, 0]
              for k, (l, _t) in enumerate(slots)]
    yield w
    w.close()
    del w
    torch.cuda.empty_cache()


def _skip(g, path):
    if g.gpir_num_variants(path) == 0:
        pytest.skip("path not built")


@pytest.mark.parametrize("path,variant", RUNS, ids=lambda x: str(x))
def test_oracle_on_64_spread_slot_groups(g, work, path, variant):
    from tests.gpu_util import to_host
    _skip(g, path)
    out = work.run(work.ct1, path, variant)
    for k, (l, t) in enumerate(work.slots):
        got = to_host(out[:, :, :, l, t].contiguous())
        assert np.array_equal(got, work.want[k]), "slot (%d, %d)" % (l, t)


@pytest.mark.parametrize("path,variant", RUNS, ids=lambda x: str(x))
def test_linearity_every_output(g, work, path, variant):
    import torch
    _skip(g, path)
    o1 = work.run(work.ct1, path, variant)
    o2 = work.run(work.ct2, path, variant)
    o3 = work.run(work.ct3, path, variant)
    bad = 0
    for c in range(work.B):
        s = o1[c] + o2[c]
        s = s - work.q32 * (s >= work.q32).to(torch.int32)
        bad += int((s != o3[c]).sum().item())
        bad += int(((o3[c] < 0) | (o3[c] >= work.q32)).sum().item())   # canonical outputs
    assert bad == 0, "%d outputs violate linearity or range" % bad


@pytest.mark.parametrize("path,variant", RUNS, ids=lambda x: str(x))
def test_toy_rlwe_one_hot_every_output(g, work, path, variant):
    _skip(g, path)
    out = work.run(work.ctq, path, variant)
    q64 = work.q32.long()
    bad = 0
    for c in range(work.B):
        a = out[c, :, 0].long()
        b = out[c, :, 1].long()
        m = (b - (a * work.sec[c].long().unsqueeze(0)) % q64) % q64
        bad += int((m != work.db[work.istar[c]].long()).sum().item())
    assert bad == 0, "%d outputs do not decrypt to the selected row" % bad
