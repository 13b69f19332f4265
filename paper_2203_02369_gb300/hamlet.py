"""Python face of libhamlet: problems and chain states over torch tensors.

PyTorch supplies device memory and the current CUDA stream; every step of the
posterior, its gradient and the HMC chain runs in libhamlet's kernels.
"""
from __future__ import annotations

import ctypes as ct
from dataclasses import asdict

import numpy as np
import torch

from . import _lib
from ._lib import HamletError, check
from .mock import Cosmology, MockSpec

_FT = {0: torch.float32, 1: torch.float64}
_CT = {0: torch.complex64, 1: torch.complex128}


def _ptr(t):
    return ct.c_void_p(t.data_ptr()) if t is not None else ct.c_void_p(0)


def _stream():
    return ct.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(a):
    return a.ctypes.data_as(_lib.c_double_p)


class Problem:
    """One reconstruction problem: grid, cosmology, catalogue, distance prior.

    prior: None or ("dz", bin_width, pad): eq. D from the redshifts of each
    catalogue set (section "Priors"; bin_width <= 0: 5 Mpc/h, pad <= 0:
    3 sigma_v/H0); ("table", d0, bin_width, logdens); ("power", alpha, dmin, dmax).
    """

    def __init__(self, N, L, cosmo=None, sigma_nl=250.0, precision="fp32", prior=None,
                 observer=None, device=0):
        self.lib = _lib.load()
        cosmo = cosmo or Cosmology()
        c = asdict(cosmo) if isinstance(cosmo, Cosmology) else dict(cosmo)
        d = _lib.hm_problem_desc()
        d.N = int(N)
        d.precision = 0 if precision == "fp32" else 1
        d.L = float(L)
        if observer is not None:
            d.observer_set = 1
            for j in range(3):
                d.observer[j] = float(observer[j])
        d.omega_m = c.get("omega_m", 0.3)
        d.omega_b = c.get("omega_b", 0.05)
        d.h = c.get("h", 0.7)
        d.n_s = c.get("n_s", 0.96)
        d.sigma8 = c.get("sigma8", 0.8)
        d.T_cmb = c.get("T_cmb", 2.7255)
        d.f_growth = c.get("f_growth", -1.0)
        d.sigma_nl = float(sigma_nl)
        prior = prior or ("dz", 0.0, 0.0)
        self._prior_keep = None
        if prior[0] == "dz":
            d.prior_kind = _lib.HM_PRIOR_DZ
            d.prior_bin = float(prior[1])
            d.prior_pad = float(prior[2])
        elif prior[0] == "table":
            d.prior_kind = _lib.HM_PRIOR_TABLE
            d.prior_d0 = float(prior[1])
            d.prior_bin = float(prior[2])
            ld = np.ascontiguousarray(prior[3], dtype=np.float64)
            self._prior_keep = ld
            d.prior_nbins = ld.shape[0]
            d.prior_logdens_host = _dptr(ld)
        else:
            d.prior_kind = _lib.HM_PRIOR_POWER
            d.prior_alpha, d.prior_dmin, d.prior_dmax = map(float, prior[1:4])
        d.device = int(device)
        self.N = int(N)
        self.L = float(L)
        self.prec = d.precision
        self.device = torch.device("cuda", int(device))
        self.dtype = _FT[self.prec]
        self.cdtype = _CT[self.prec]
        self.h = ct.c_void_p()
        check(self.lib.hm_init_problem(ct.byref(d), ct.byref(self.h)))
        self.n = 0

    @classmethod
    def from_mock(cls, spec: MockSpec, cat: dict, device=0, prior=None):
        """The mock's problem; the distance prior defaults to eq. D built from
        its redshifts with the spec's bin width."""
        p = cls(spec.N, spec.L, spec.cosmo, spec.sigma_nl, spec.precision, prior or ("dz", spec.prior_bin, 0.0),
                device=device)
        p.set_catalog(cat["rhat"], cat["mu"], cat["sigma_mu"], cat["cz"], cat["sigma_cz"])
        return p

    def close(self):
        if self.h:
            self.lib.hm_destroy_problem(self.h)
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_catalog(self, rhat, mu, sigma_mu, cz, sigma_cz=None):
        rhat = np.ascontiguousarray(rhat, dtype=np.float64).reshape(-1, 3)
        n = rhat.shape[0]
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (mu, sigma_mu, cz)]
        scz = None if sigma_cz is None else np.ascontiguousarray(sigma_cz, dtype=np.float64)
        check(self.lib.hm_set_catalog(self.h, n, _dptr(rhat), _dptr(arrs[0]), _dptr(arrs[1]),
                                      _dptr(arrs[2]), _dptr(scz) if scz is not None else None))
        self.n = n

    def set_catalog_sg(self, sgl_deg, sgb_deg, mu, sigma_mu, cz, sigma_cz=None):
        """The catalogue as supergalactic longitude/latitude in degrees."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (sgl_deg, sgb_deg, mu, sigma_mu, cz)]
        n = arrs[0].shape[0]
        scz = None if sigma_cz is None else np.ascontiguousarray(sigma_cz, dtype=np.float64)
        check(self.lib.hm_set_catalog_sg(self.h, n, *[_dptr(a) for a in arrs],
                                         _dptr(scz) if scz is not None else None))
        self.n = n

    @property
    def info(self):
        i = _lib.hm_problem_info()
        check(self.lib.hm_problem_get_info(self.h, ct.byref(i)))
        return {k: getattr(i, k) for k, _ in i._fields_}

    def field(self, value=None):
        t = torch.zeros((self.N,) * 3, dtype=self.dtype, device=self.device)
        if value is not None:
            t.copy_(torch.as_tensor(value))
        return t

    def logpost_grad(self, w, d):
        """(Psi, dPsi/dw, dPsi/dd) at (w, d); Psi is a 0-d float64 tensor."""
        w = w.to(self.device, self.dtype).contiguous()
        d = d.to(self.device, torch.float64).contiguous()
        psi = torch.empty((), dtype=torch.float64, device=self.device)
        gw = torch.empty_like(w)
        gd = torch.empty_like(d)
        check(self.lib.hm_logpost_grad(self.h, _ptr(w), _ptr(d), _ptr(psi), _ptr(gw), _ptr(gd), _stream()))
        return psi, gw, gd

    def logpost_grad_noalloc(self, w, d):
        """As logpost_grad, through the entry point that takes its scratch from
        the library's static device array instead of allocating any."""
        w = w.to(self.device, self.dtype).contiguous()
        d = d.to(self.device, torch.float64).contiguous()
        psi = torch.empty((), dtype=torch.float64, device=self.device)
        gw = torch.empty_like(w)
        gd = torch.empty_like(d)
        check(self.lib.hm_logpost_grad_noalloc(self.h, _ptr(w), _ptr(d), _ptr(psi), _ptr(gw), _ptr(gd),
                                               _stream()))
        return psi, gw, gd

    def prior_table(self):
        """(d0, bin width, ln pi_D at the bin centres) of the distance prior
        as the device reads it."""
        nb, d0, bw = ct.c_int32(), ct.c_double(), ct.c_double()
        check(self.lib.hm_problem_prior_table(self.h, 0, None, ct.byref(nb), ct.byref(d0), ct.byref(bw)))
        t = np.zeros(max(nb.value, 1))
        check(self.lib.hm_problem_prior_table(self.h, nb.value, _dptr(t), ct.byref(nb), None, None))
        return d0.value, bw.value, t[:nb.value].copy()

    def last_status(self):
        v = ct.c_int32()
        check(self.lib.hm_problem_last_status(self.h, _stream(), ct.byref(v)))
        return v.value

    def velocity_field(self, w):
        w = w.to(self.device, self.dtype).contiguous()
        v = torch.empty((3,) + (self.N,) * 3, dtype=self.dtype, device=self.device)
        check(self.lib.hm_velocity_field(self.h, _ptr(w), _ptr(v), _stream()))
        return v

    def fft_r2c(self, x):
        x = x.to(self.device, self.dtype).contiguous()
        cnt = x.numel() // self.N ** 3
        out = torch.empty((cnt, self.N, self.N, self.N // 2 + 1), dtype=self.cdtype, device=self.device)
        check(self.lib.hm_fft_r2c(self.h, _ptr(x), _ptr(out), cnt, _stream()))
        return out

    def fft_c2r(self, X):
        X = X.to(self.device, self.cdtype).contiguous()
        cnt = X.numel() // (self.N * self.N * (self.N // 2 + 1))
        out = torch.empty((cnt,) + (self.N,) * 3, dtype=self.dtype, device=self.device)
        check(self.lib.hm_fft_c2r(self.h, _ptr(X), _ptr(out), cnt, _stream()))
        return out

    def cells(self, d, sort=True):
        d = d.to(self.device, torch.float64).contiguous()
        cell = torch.empty(d.shape[0], dtype=torch.int32, device=self.device)
        perm = torch.empty(d.shape[0], dtype=torch.int32, device=self.device) if sort else None
        check(self.lib.hm_cells(self.h, _ptr(d), _ptr(cell), _ptr(perm), _stream()))
        return cell, perm


TRACE_DTYPE = np.dtype([("traj", np.int64), ("H_old", np.float64), ("H_new", np.float64),
                        ("logu", np.float64), ("psi", np.float64), ("eps", np.float64), ("accept", np.int32),
                        ("status", np.int32)])


class State:
    """n_chains HMC chains over one or several problems of the same grid."""

    def __init__(self, problems, d_init, seed=0, chain_problem=None, chain_ids=None):
        if isinstance(problems, Problem):
            problems = [problems]
        self.problems = list(problems)
        self.lib = self.problems[0].lib
        nch = len(d_init)
        self.C = nch
        cp = list(chain_problem) if chain_problem is not None else [0] * nch
        self.chain_problem = cp
        self._d = [np.ascontiguousarray(x, dtype=np.float64) for x in d_init]
        harr = (ct.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        cparr = (ct.c_int32 * nch)(*cp)
        idarr = (ct.c_int32 * nch)(*(chain_ids if chain_ids is not None else range(nch)))
        darr = (_lib.c_double_p * nch)(*[_dptr(x) for x in self._d])
        self.h = ct.c_void_p()
        check(self.lib.hm_state_create_batch(harr, len(self.problems), nch, cparr, idarr,
                                             ct.c_uint64(int(seed)), darr, ct.byref(self.h)))
        p0 = self.problems[0]
        self.N, self.dtype, self.device = p0.N, p0.dtype, p0.device
        self._an_radii = None
        self.seed = int(seed)
        self.chain_ids = list(chain_ids) if chain_ids is not None else list(range(nch))
        self._sig_on = False

    def close(self):
        if self.h:
            self.lib.hm_destroy_state(self.h)
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _n(self, c):
        return self.problems[self.chain_problem[c]].n

    def set(self, chain=0, w=None, d=None, pw=None, pd=None):
        """Copy a chain's position and/or momenta in.  Device tensors, or host
        tensors (pinned ones are copied asynchronously on the current stream;
        the state keeps a reference to them until the next set)."""
        def conv(t, dt):
            if t is None:
                return None
            if t.device.type == "cpu":
                return t.to(dt).contiguous()
            return t.to(self.device, dt).contiguous()
        w, pw = conv(w, self.dtype), conv(pw, self.dtype)
        d, pd = conv(d, torch.float64), conv(pd, torch.float64)
        check(self.lib.hm_state_set(self.h, chain, _ptr(w), _ptr(d), _ptr(pw), _ptr(pd), _stream()))
        self._keep = (w, d, pw, pd)

    def get(self, chain=0, out=None):
        """A chain's position and momenta as new device tensors, or, with out
        (a dict of contiguous tensors keyed by some of "w", "d", "pw", "pd", on
        the device or on the host), copied into those only (asynchronous on
        the current stream for device and pinned host tensors)."""
        if out is not None:
            want = {"w": self.dtype, "pw": self.dtype, "d": torch.float64, "pd": torch.float64}
            size = {"w": self.N ** 3, "pw": self.N ** 3, "d": self._n(chain), "pd": self._n(chain)}
            for k, t in out.items():
                if k not in want or t.dtype != want[k] or not t.is_contiguous() or t.numel() != size[k]:
                    raise ValueError(f"out[{k!r}] must be a contiguous {want.get(k)} tensor of {size.get(k)} "
                                     "elements")
            p = {k: (_ptr(out[k]) if k in out else None) for k in want}
            check(self.lib.hm_state_get(self.h, chain, p["w"], p["d"], p["pw"], p["pd"], _stream()))
            return out
        N = self.N
        w = torch.empty((N,) * 3, dtype=self.dtype, device=self.device)
        pw = torch.empty_like(w)
        n = self._n(chain)
        d = torch.empty(n, dtype=torch.float64, device=self.device)
        pd = torch.empty_like(d)
        check(self.lib.hm_state_get(self.h, chain, _ptr(w), _ptr(d), _ptr(pw), _ptr(pd), _stream()))
        return dict(w=w, d=d, pw=pw, pd=pd)

    def grad(self, chain=0):
        gw = torch.empty((self.N,) * 3, dtype=self.dtype, device=self.device)
        gd = torch.empty(self._n(chain), dtype=torch.float64, device=self.device)
        check(self.lib.hm_state_get_grad(self.h, chain, _ptr(gw), _ptr(gd), _stream()))
        return gw, gd

    def refresh(self):
        check(self.lib.hm_state_refresh(self.h, _stream()))

    def scalars(self, chain=0):
        psi, kin, traj = ct.c_double(), ct.c_double(), ct.c_int64()
        check(self.lib.hm_state_scalars(self.h, chain, ct.byref(psi), ct.byref(kin), ct.byref(traj), _stream()))
        return dict(psi=psi.value, kinetic=kin.value, traj=traj.value)

    def set_traj(self, chain, traj):
        check(self.lib.hm_state_set_traj(self.h, chain, int(traj)))

    def profile(self, enable=True):
        check(self.lib.hm_state_profile(self.h, int(bool(enable))))

    def profile_collect(self):
        check(self.lib.hm_state_profile_collect(self.h))

    def profile_read(self):
        """{kernel kind: (total ms, launches)} accumulated by run_chain."""
        nk = ct.c_int32()
        ms = (ct.c_double * 64)()
        ln = (ct.c_int64 * 64)()
        check(self.lib.hm_state_profile_read(self.h, 64, ms, ln, ct.byref(nk)))
        return {self.lib.hm_kernel_kind_name(k).decode(): (ms[k], ln[k]) for k in range(nk.value)}

    # -- checkpoint / resume ------------------------------------------------
    # A chain is resumed exactly by its position (w, d; sigma_NL when it is
    # sampled) and its trajectory counter: the momenta are drawn afresh at the
    # start of every trajectory from Philox counters (element pair,
    # trajectory, chain word, tag) under the state's key, so the continued
    # chain draws the numbers the uninterrupted one would have drawn.
    # File layout (little endian): 8-byte magic, int32 version, N, precision
    # (0 FP32, 1 FP64), sigma_NL sampled flag; int64 n points, trajectory
    # counter, Philox key, chain word; float64 sigma_NL; then w (N^3 values of
    # the field precision) and d (n float64).
    CHECKPOINT_MAGIC = b"HMCHAIN\x01"
    _HDR = "<8siiiiqqqqd"

    def save(self, path, chain=0):
        """Write chain `chain`'s resumable state to a host file."""
        import struct
        g = self.get(chain)
        traj = self.scalars(chain)["traj"]
        sig = float(self.sigma_nl()[0][chain]) if self._sig_on else 0.0
        prec = 0 if self.dtype == torch.float32 else 1
        hdr = struct.pack(self._HDR, self.CHECKPOINT_MAGIC, 1, self.N, prec, int(self._sig_on), self._n(chain),
                          int(traj), self.seed, int(self.chain_ids[chain]), sig)
        with open(path, "wb") as fh:
            fh.write(hdr)
            fh.write(g["w"].cpu().numpy().tobytes())
            fh.write(g["d"].cpu().numpy().astype(np.float64).tobytes())

    def restore(self, path, chain=0):
        """Load a state written by save() into chain `chain` (same grid,
        precision, catalogue size, Philox key and chain word), set its
        trajectory counter and re-evaluate Psi and the gradient there."""
        import struct
        with open(path, "rb") as fh:
            raw = fh.read()
        hs = struct.calcsize(self._HDR)
        magic, ver, N, prec, sig_on, n, traj, seed, cid, sig = struct.unpack(self._HDR, raw[:hs])
        if magic != self.CHECKPOINT_MAGIC or ver != 1:
            raise HamletError(-1, f"{path}: not a chain checkpoint")
        mine = 0 if self.dtype == torch.float32 else 1
        if (N, prec, n) != (self.N, mine, self._n(chain)):
            raise HamletError(-1, f"{path}: grid/precision/points {(N, prec, n)} differ from the chain's "
                                  f"{(self.N, mine, self._n(chain))}")
        if (seed, cid) != (self.seed, int(self.chain_ids[chain])):
            raise HamletError(-1, f"{path}: Philox key/chain word {(seed, cid)} differ from the chain's "
                                  f"{(self.seed, int(self.chain_ids[chain]))}: it would not continue its stream")
        esz = 4 if prec == 0 else 8
        nw = N ** 3 * esz
        if len(raw) != hs + nw + 8 * n:
            raise HamletError(-1, f"{path}: truncated checkpoint")
        w = np.frombuffer(raw, dtype=np.float32 if prec == 0 else np.float64, count=N ** 3, offset=hs)
        d = np.frombuffer(raw, dtype=np.float64, count=n, offset=hs + nw)
        self.set(chain, w=torch.tensor(w.reshape((N,) * 3).copy()), d=torch.tensor(d.copy()))
        self.set_traj(chain, traj)
        if sig_on:
            cur = self.sigma_nl()[0] if self._sig_on else np.full(self.C, sig)
            cur[chain] = sig
            self.sample_sigma_nl(True, cur)
        else:
            self.refresh()

    def sample_sigma_nl(self, enable=True, sigma0=None):
        self._sig_on = bool(enable)
        s0 = None if sigma0 is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(sigma0, dtype=np.float64), (self.C,)))
        check(self.lib.hm_state_sample_sigma_nl(self.h, int(bool(enable)), _dptr(s0) if s0 is not None else None,
                                                _stream()))

    def sigma_nl(self):
        """(current sigma_NL per chain, dPsi/dsigma_NL per chain)."""
        s = np.zeros(self.C)
        g = np.zeros(self.C)
        check(self.lib.hm_state_get_sigma_nl(self.h, _dptr(s), _dptr(g), _stream()))
        return s, g

    def analytics(self, enable=True, radii=(), max_samples=1024):
        """Turn the on-device chain analytics on (zeroed) or off; radii of the
        spheres about the observer for the monopole and dipole."""
        r = np.ascontiguousarray(radii, dtype=np.float64)
        check(self.lib.hm_state_analytics(self.h, int(bool(enable)), int(r.shape[0]), _dptr(r) if r.size else None,
                                          int(max_samples), _stream()))
        self._an_radii = r.copy() if enable else None
        self._an_max = int(max_samples)

    def analytics_read(self, chain=0, max_metric=None):
        """Mean/variance fields of delta and v_r, the convergence values and
        the sphere moments (mean, variance over samples) of one chain."""
        dt = self.dtype
        shape = (self.N,) * 3
        md, vd, mv, vv = (torch.empty(shape, dtype=dt, device=self.device) for _ in range(4))
        if self._an_radii is None:
            raise HamletError(-5, "chain analytics are off (State.analytics)")
        nr = self._an_radii.shape[0]
        if max_metric is None:
            max_metric = self._an_max
        met = np.zeros(max(1, max_metric))
        sph = np.zeros((max(nr, 1), 5, 2))
        n = ct.c_int64()
        check(self.lib.hm_state_analytics_read(self.h, int(chain), _ptr(md), _ptr(vd), _ptr(mv), _ptr(vv),
                                               _dptr(met), int(max_metric), _dptr(sph), ct.byref(n), _stream()))
        ns = n.value
        return {"n_samples": ns, "mean_delta": md, "var_delta": vd, "mean_vr": mv, "var_vr": vv,
                "metric": met[:max(0, min(ns - 1, max_metric))].copy(), "sphere": sph[:nr].copy()}

    def adapt_step_size(self, n_warmup, n_leapfrog, eps0, target=0.65, sample_distances=True):
        """Dual-averaging warm-up; returns (tuned eps per chain, trace)."""
        e0 = np.ascontiguousarray(np.broadcast_to(np.asarray(eps0, dtype=np.float64), (self.C,)))
        eo = np.zeros(self.C)
        tr = (_lib.hm_trace * (max(n_warmup, 1) * self.C))()
        check(self.lib.hm_adapt_step_size(self.h, int(n_warmup), int(n_leapfrog), float(target), _dptr(e0),
                                          int(bool(sample_distances)), _dptr(eo), tr, _stream()))
        out = np.frombuffer(tr, dtype=TRACE_DTYPE, count=n_warmup * self.C).copy()
        return eo, out.reshape(n_warmup, self.C)

    def leapfrog(self, n_steps, eps, sample_distances=True):
        check(self.lib.hm_leapfrog(self.h, int(n_steps), float(eps), int(bool(sample_distances)), _stream()))

    def run_chain(self, n_traj, n_leapfrog, eps, sample_distances=True, use_graph=False, trace=True):
        eps_arr = np.ascontiguousarray(np.broadcast_to(np.asarray(eps, dtype=np.float64), (self.C,)))
        tr = (_lib.hm_trace * (max(n_traj, 1) * self.C))() if trace else None
        check(self.lib.hm_run_chain(self.h, int(n_traj), int(n_leapfrog), _dptr(eps_arr),
                                    int(bool(sample_distances)), int(bool(use_graph)), tr, _stream()))
        if not trace:
            return None
        out = np.frombuffer(tr, dtype=TRACE_DTYPE, count=n_traj * self.C).copy()
        return out.reshape(n_traj, self.C)


class Slots:
    """Slotted state for continuous batching: up to n_slots jobs of one grid
    (the template's N, precision, box and P(k)) advance together, each
    trajectory of every loaded job in the same kernel launches.  Jobs are
    loaded and released between trajectories; loaded chains are packed at
    indices 0..n_active-1 (a release moves the last one into the freed
    index, which release() reports)."""

    def __init__(self, template, n_slots, max_points, seed=0):
        self.lib = template.lib
        self.template = template
        self.N, self.dtype, self.device = template.N, template.dtype, template.device
        self.h = ct.c_void_p()
        check(self.lib.hm_slots_create(template.h, int(n_slots), int(max_points), ct.c_uint64(int(seed)),
                                       ct.byref(self.h)))
        self.n_slots = int(n_slots)
        self.max_points = int(max_points)
        self.problems = []      # problem of each loaded index (the library reads its prior in place)
        self._keep = []

    def close(self):
        if self.h:
            self.lib.hm_destroy_state(self.h)
            self.h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_active(self):
        a, n = ct.c_int32(), ct.c_int32()
        check(self.lib.hm_slots_count(self.h, ct.byref(a), ct.byref(n)))
        return a.value

    def load(self, problem, d_init, chain_id, eps0, adapt_target=0.0, sigma_nl0=0.0):
        """Load a job; returns its chain index.  sigma_nl0 > 0: the job samples
        sigma_NL starting there."""
        d = np.ascontiguousarray(d_init, dtype=np.float64)
        idx = ct.c_int32()
        check(self.lib.hm_slots_load(self.h, problem.h, int(chain_id), _dptr(d) if d.size else None,
                                     float(eps0), float(adapt_target), float(sigma_nl0), ct.byref(idx),
                                     _stream()))
        assert idx.value == len(self.problems)
        self.problems.append(problem)
        return idx.value

    def adapt_end(self, index):
        e = np.zeros(1)
        check(self.lib.hm_slots_adapt_end(self.h, int(index), _dptr(e), _stream()))
        return float(e[0])

    def release(self, index):
        """Release a job; returns the old index of the chain now at `index`
        (-1 if none moved)."""
        mv = ct.c_int32()
        check(self.lib.hm_slots_release(self.h, int(index), ct.byref(mv), _stream()))
        last = self.problems.pop()
        if mv.value >= 0:
            self.problems[index] = last
        return mv.value

    def run(self, n_traj=1, n_leapfrog=20, use_graph=True):
        """n_traj trajectories of every loaded job; trace [n_traj, n_active]."""
        na = len(self.problems)
        tr = (_lib.hm_trace * (max(n_traj, 1) * max(na, 1)))()
        check(self.lib.hm_slots_run(self.h, int(n_traj), int(n_leapfrog), int(bool(use_graph)), tr, _stream()))
        out = np.frombuffer(tr, dtype=TRACE_DTYPE, count=n_traj * na).copy()
        return out.reshape(n_traj, na)

    def get(self, index):
        w = torch.empty((self.N,) * 3, dtype=self.dtype, device=self.device)
        pw = torch.empty_like(w)
        n = self.problems[index].n
        d = torch.empty(n, dtype=torch.float64, device=self.device)
        pd = torch.empty_like(d)
        check(self.lib.hm_state_get(self.h, int(index), _ptr(w), _ptr(d), _ptr(pw), _ptr(pd), _stream()))
        return dict(w=w, d=d, pw=pw, pd=pd)

    def grad(self, index):
        gw = torch.empty((self.N,) * 3, dtype=self.dtype, device=self.device)
        gd = torch.empty(self.problems[index].n, dtype=torch.float64, device=self.device)
        check(self.lib.hm_state_get_grad(self.h, int(index), _ptr(gw), _ptr(gd), _stream()))
        return gw, gd

    def sigma_nl(self):
        """(sigma_NL, dPsi/dsigma_NL) of every loaded chain."""
        na = len(self.problems)
        s, g = np.zeros(max(na, 1)), np.zeros(max(na, 1))
        check(self.lib.hm_state_get_sigma_nl(self.h, _dptr(s), _dptr(g), _stream()))
        return s[:na], g[:na]

    def scalars(self, index):
        psi, kin, traj = ct.c_double(), ct.c_double(), ct.c_int64()
        check(self.lib.hm_state_scalars(self.h, int(index), ct.byref(psi), ct.byref(kin), ct.byref(traj),
                                        _stream()))
        return dict(psi=psi.value, kinetic=kin.value, traj=traj.value)


def philox(seed, n, c1, c2, c3, device=0):
    lib = _lib.load()
    out = torch.empty(4 * n, dtype=torch.int32, device=torch.device("cuda", device))
    check(lib.hm_philox(ct.c_uint64(int(seed)), int(n), c1, c2, c3, _ptr(out), _stream()))
    return out.view(torch.int32)


def dz_prior_table(cz, omega_m=0.3, bin_width=5.0, pad=10.0):
    """ln density table of the redshift-distance histogram prior (eq. D),
    computed by libhamlet on the host; use as ("table", 0.0, bin_width, table)."""
    lib = _lib.load()
    cz = np.ascontiguousarray(cz, dtype=np.float64)
    nb = ct.c_int32()
    lib.hm_dz_prior_table(float(omega_m), cz.shape[0], _dptr(cz), float(bin_width), float(pad), 0, None,
                          ct.byref(nb))
    out = np.zeros(nb.value)
    check(lib.hm_dz_prior_table(float(omega_m), cz.shape[0], _dptr(cz), float(bin_width), float(pad), nb.value,
                                _dptr(out), ct.byref(nb)))
    return out
