"""Python front end of libaxpic: owns the particle slabs as torch CUDA tensors
and forwards every operator to the C ABI. PyTorch provides device memory and
the stream; all arithmetic of the method runs in the library's kernels.
"""
import ctypes

import numpy as np
import torch

from . import _lib

SPECIES = ("electrons", "photons", "axions")
FIELDS = ("w", "px", "py", "pz", "x", "y", "z")


class SpeciesSlab:
    """Cell-sorted slab of one species, ncells * capacity slots: the records
    {w, px, py, pz} (storage["wp"]) and {x, y, z, unused} (storage["xyz"]) of
    the slots, 4 binary32 values each. data[f] is a (strided) view of field f
    over the slots."""

    def __init__(self, ncells, capacity, device):
        self.capacity = capacity
        n = max(ncells * capacity, 4)
        self.storage = {k: torch.zeros(4 * n, dtype=torch.float32, device=device) for k in ("wp", "xyz")}
        rec, pos = self.storage["wp"].view(n, 4), self.storage["xyz"].view(n, 4)
        self.data = {f: rec[:, k] for k, f in enumerate(("w", "px", "py", "pz"))}
        self.data.update({f: pos[:, k] for k, f in enumerate(("x", "y", "z"))})
        self.count = torch.zeros(max(ncells, 1), dtype=torch.int32, device=device)

    def struct(self):
        s = _lib.Species()
        for f in ("wp", "xyz"):
            setattr(s, f, self.storage[f].data_ptr())
        s.count = self.count.data_ptr()
        s.capacity = self.capacity
        return s

    def cell(self, c):
        """Host copy of cell c's particles as a dict of float64 numpy arrays."""
        n = int(self.count[c].item())
        b = c * self.capacity
        return {f: self.data[f][b:b + n].double().cpu().numpy() for f in FIELDS}

    def set_cell(self, c, arrays):
        n = len(arrays["w"])
        if n > self.capacity:
            raise ValueError("too many particles for the slab")
        b = c * self.capacity
        for f in FIELDS:
            self.data[f][b:b + n] = torch.as_tensor(np.asarray(arrays[f]), dtype=torch.float32)
        self.count[c] = n


class AxionPlasma:
    """One plasma context (axpic_init_plasma) with its slabs.

    T_keV: scalar or [ncells]; n_ion: [ncells, nspecies] in cm^-3; Z, A:
    [nspecies]; caps: (electrons, photons, axions) slots per cell; params: a
    dict of axpic_params fields overriding axpic_default_params.
    """

    def __init__(self, ncells, T_keV, n_ion, Z, A, volume_cm3, caps, params=None, device="cuda:0",
                 cell_index_base=0, stream=None):
        self.device = torch.device(device)
        self.ncells = ncells
        self.Z = np.asarray(Z, dtype=np.float64)
        self.A = np.asarray(A, dtype=np.float64)
        ns = len(self.Z)
        T = np.broadcast_to(np.asarray(T_keV, dtype=np.float64), (ncells,))
        n_ion = np.asarray(n_ion, dtype=np.float64).reshape(ncells, ns) if ncells else np.zeros((0, ns))
        self.T = torch.tensor(np.array(T), dtype=torch.float64, device=self.device)
        self.n_ion = torch.tensor(n_ion, dtype=torch.float64, device=self.device).reshape(-1)
        if self.T.numel() == 0:
            self.T = torch.zeros(1, dtype=torch.float64, device=self.device)
            self.n_ion = torch.zeros(ns, dtype=torch.float64, device=self.device)
        self.slabs = {name: SpeciesSlab(ncells, cap, self.device) for name, cap in zip(SPECIES, caps)}
        self.params = _lib.default_params()
        for k, v in (params or {}).items():
            setattr(self.params, k, v)
        self._Zc = (ctypes.c_double * ns)(*self.Z)
        self._Ac = (ctypes.c_double * ns)(*self.A)
        d = _lib.PlasmaDesc()
        d.ncells = ncells
        d.nspecies = ns
        d.cell_index_base = cell_index_base
        d.T_keV = self.T.data_ptr()
        d.n_ion = self.n_ion.data_ptr()
        d.Z = self._Zc
        d.A = self._Ac
        d.cell_volume_cm3 = volume_cm3
        d.electrons = self.slabs["electrons"].struct()
        d.photons = self.slabs["photons"].struct()
        d.axions = self.slabs["axions"].struct()
        self.desc = d
        self.volume = volume_cm3
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.ctx = _lib.axpic_init_plasma(d, self.params, self.stream.cuda_stream)
        self.nbins = self.params.tally_nbins

    # -------------------------------------------------------------- operators
    def sample(self, n_el, n_ph, n_ax=0):
        _lib.axpic_sample_plasma(self.ctx, n_el, n_ph, n_ax)

    def update_cells(self):
        _lib.axpic_update_cells(self.ctx)

    def absorb(self, step, mask=_lib.CH_ALL):
        _lib.axpic_absorb(self.ctx, step, mask)

    def emit(self, step, mask=_lib.CH_ALL):
        _lib.axpic_emit(self.ctx, step, mask)

    def feedback(self, step):
        _lib.axpic_feedback(self.ctx, step)

    def step(self, step, mask=_lib.CH_ALL):
        _lib.axpic_step(self.ctx, step, mask)

    def step_cells(self, step, first_cell, ncells, mask=_lib.CH_ALL):
        """One full step over cells [first_cell, first_cell + ncells) only
        (axpic_step_cells); asynchronous."""
        _lib.axpic_step_cells(self.ctx, step, mask, first_cell, ncells)

    def run_steps(self, first_step, nsteps, mask=_lib.CH_ALL):
        """nsteps full steps by replaying a CUDA graph of one step."""
        _lib.axpic_run_steps(self.ctx, first_step, nsteps, mask)

    def launch_shape(self):
        """(decide_chunk, event warps per CTA, branches of a replayed step)."""
        return _lib.axpic_launch_shape(self.ctx)

    def autotune(self, step, trial_steps=3, mask=_lib.CH_ALL):
        """Times the launch shapes on this state (restored afterwards) and keeps
        the fastest; returns (ms per step, decide_chunk, event warps)."""
        return _lib.axpic_autotune(self.ctx, step, trial_steps, mask)

    def tally(self):
        """(H [3, nbins] keV-weighted histogram, totals dict); clears the tally."""
        H = (ctypes.c_double * (3 * self.nbins))()
        T = (ctypes.c_double * _lib.TOTALS_LEN)()
        _lib.axpic_tally_spectrum(self.ctx, self.nbins, H, T)
        return np.array(H).reshape(3, self.nbins), dict(zip(_lib.TOTALS_NAMES, list(T)))

    def eval_rates(self, cell, E_keV):
        E = torch.as_tensor(np.asarray(E_keV), dtype=torch.float32, device=self.device).contiguous()
        out = torch.empty(4 * max(E.numel(), 1), dtype=torch.float32, device=self.device)
        _lib.axpic_eval_rates(self.ctx, cell, E.data_ptr(), E.numel(), out.data_ptr())
        self.stream.synchronize()
        return out[:4 * E.numel()].reshape(-1, 4).double().cpu().numpy()

    def cell_info(self, first=0, count=None):
        count = self.ncells - first if count is None else count
        buf = (ctypes.c_double * (_lib.CELL_INFO_LEN * max(count, 1)))()
        _lib.axpic_get_cell_info(self.ctx, first, count, buf)
        return np.array(buf)[:_lib.CELL_INFO_LEN * count].reshape(count, _lib.CELL_INFO_LEN)

    def cell_diag(self, first=0, count=None):
        count = self.ncells - first if count is None else count
        buf = (ctypes.c_double * (_lib.CELL_DIAG_LEN * max(count, 1)))()
        _lib.axpic_get_cell_diag(self.ctx, first, count, buf)
        return np.array(buf)[:_lib.CELL_DIAG_LEN * count].reshape(count, _lib.CELL_DIAG_LEN)

    def residuals(self, first=0, count=None):
        count = self.ncells - first if count is None else count
        buf = (ctypes.c_double * (4 * max(count, 1)))()
        _lib.axpic_get_residuals(self.ctx, first, count, buf)
        return np.array(buf)[:4 * count].reshape(count, 4)

    def stream_axions(self, dims, h_cm, dt_s, periodic=True, mass_keV=0.0):
        """Axion free streaming and cell migration on an nx x ny x nz grid
        (axpic_stream_axions); mass_keV: the axion mass (0: massless, at c);
        asynchronous."""
        _lib.axpic_stream_axions(self.ctx, dims, h_cm, dt_s, 0 if periodic else 1, mass_keV)

    def run_steps_streamed(self, first, nsteps, mask, dims, h_cm, dt_s, periodic=True, mass_keV=0.0):
        """nsteps steps, each followed by the axions' streaming, replayed from
        CUDA graphs (axpic_run_steps_streamed); asynchronous."""
        _lib.axpic_run_steps_streamed(self.ctx, first, nsteps, mask, dims, h_cm, dt_s, 0 if periodic else 1,
                                      mass_keV)

    def deposit_composition(self, mass_frac=None, bind_species=-1, out=None):
        """Ion densities from the deposited electron density
        (axpic_deposit_composition): mass fractions under quasi-neutrality, or
        the whole density on bind_species. out: a device float64 tensor of
        ncells * nspecies (default: the context's own n_ion, whose records are
        then rebuilt); asynchronous; returns out."""
        out = self.n_ion if out is None else out
        _lib.axpic_deposit_composition(self.ctx, bind_species, mass_frac, out.data_ptr())
        return out

    def merge_axions(self, n_target, edges_p2):
        """Merging of the axions of every cell above n_target (axpic_merge_axions);
        edges_p2: ascending |p|^2 thresholds in (m_e c)^2; asynchronous."""
        _lib.axpic_merge_axions(self.ctx, n_target, edges_p2)

    def merge_stats(self):
        """Axions removed by merging so far."""
        return _lib.axpic_merge_stats(self.ctx)

    def save_state(self):
        """The library-owned state (axpic_save_state) as a uint8 array; the
        slabs and T are the caller's (this object's tensors)."""
        return _lib.axpic_save_state(self.ctx)

    def load_state(self, buf):
        """Loads a save_state array into this context (axpic_load_state)."""
        _lib.axpic_load_state(self.ctx, buf)

    def stream_stats(self):
        """[escaped number, escaped weight, escaped weight x energy (keV),
        dropped number] over every streaming call so far."""
        return _lib.axpic_stream_stats(self.ctx)

    def profile_begin(self, max_steps):
        _lib.axpic_profile_begin(self.ctx, max_steps)

    def profile_end(self):
        return _lib.axpic_profile_end(self.ctx)

    def sync(self):
        _lib.axpic_sync(self.ctx)

    def close(self):
        if self.ctx is not None:
            ctx, self.ctx = self.ctx, None
            _lib.axpic_destroy(ctx)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------------- host views
    def cell(self, c):
        """Host copy of cell c: {'e': ..., 'g': ..., 'a': ...} dicts of arrays."""
        return {k: self.slabs[name].cell(c) for k, name in zip("ega", SPECIES)}

    def set_cell(self, c, parts):
        for k, name in zip("ega", SPECIES):
            if k in parts:
                self.slabs[name].set_cell(c, parts[k])

    def counts(self):
        return {name: self.slabs[name].count[:self.ncells].cpu().numpy() for name in SPECIES}

    def temperatures(self):
        return self.T[:self.ncells].cpu().numpy()
