"""Thin Python binding over the C ABI of libpm (include/pm.h).

Every function here marshals arguments and calls one library entry point;
torch supplies device memory and the current CUDA stream.  All arithmetic
of the PM step runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Dict, Optional, Sequence, Tuple

import torch

from . import _lib
from ._lib import pm_codes_t, pm_config_t, pm_particles_t, pm_tuning_t


class PMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Codes:
    """One species' compressed state in device memory (layout of pm_codes_t)."""
    n: int
    cnt: torch.Tensor       # uint8 [n_cmp^3]
    esc: torch.Tensor       # int32 viewed as uint32 pairs [esc_cap, 2]
    n_esc: torch.Tensor     # int32 [1]
    pos: torch.Tensor       # uint8 [n, 4]: px, py, pz, 0
    vel: torch.Tensor       # int16 (uint16 bits) or uint8 [n, 4]: vx, vy, vz, 0
    vmax: torch.Tensor      # float32 [1]

    @staticmethod
    def empty(n: int, n_cmp: int, vel_bits: int, esc_cap: Optional[int] = None, device="cuda") -> "Codes":
        ncell = n_cmp ** 3
        if esc_cap is None:
            esc_cap = max(1, min(ncell, n // 255 + 1))
        vdt = torch.int16 if vel_bits == 16 else torch.uint8
        return Codes(n=n, cnt=torch.empty(ncell, dtype=torch.uint8, device=device),
                     esc=torch.zeros((esc_cap, 2), dtype=torch.int32, device=device),
                     n_esc=torch.zeros(1, dtype=torch.int32, device=device),
                     pos=torch.zeros((n, 4), dtype=torch.uint8, device=device),
                     vel=torch.zeros((n, 4), dtype=vdt, device=device),
                     vmax=torch.zeros(1, dtype=torch.float32, device=device))

    @staticmethod
    def empty_packed(n: int, n_cmp: int, vel_bits: int, esc_cap: Optional[int] = None, device="cuda") -> "Codes":
        """Packed form: pos uint8 [n, 3], vel uint8 or int16 (u16 bits) [n, 3]."""
        ncell = n_cmp ** 3
        if esc_cap is None:
            esc_cap = max(1, min(ncell, n // 255 + 1))
        vdt = torch.int16 if vel_bits == 16 else torch.uint8
        return Codes(n=n, cnt=torch.empty(ncell, dtype=torch.uint8, device=device),
                     esc=torch.zeros((esc_cap, 2), dtype=torch.int32, device=device),
                     n_esc=torch.zeros(1, dtype=torch.int32, device=device),
                     pos=torch.zeros((n, 3), dtype=torch.uint8, device=device),
                     vel=torch.zeros((n, 3), dtype=vdt, device=device),
                     vmax=torch.zeros(1, dtype=torch.float32, device=device))

    def struct(self) -> pm_codes_t:
        return pm_codes_t(self.n, self.cnt.data_ptr(), self.esc.data_ptr(), self.esc.shape[0],
                          self.n_esc.data_ptr(), self.pos.data_ptr(), self.vel.data_ptr(), self.vmax.data_ptr())

    def to(self, device, pin: bool = False) -> "Codes":
        def mv(t):
            out = t.to(device)
            return out.pin_memory() if pin and out.device.type == "cpu" else out
        return Codes(self.n, mv(self.cnt), mv(self.esc), mv(self.n_esc), mv(self.pos), mv(self.vel), mv(self.vmax))

    def clone(self) -> "Codes":
        return Codes(self.n, self.cnt.clone(), self.esc.clone(), self.n_esc.clone(), self.pos.clone(),
                     self.vel.clone(), self.vmax.clone())

    def copy_(self, src: "Codes") -> "Codes":
        """Copy src's codes into this object's buffers (same shapes), stream-ordered."""
        for name in ("cnt", "esc", "n_esc", "pos", "vel", "vmax"):
            getattr(self, name).copy_(getattr(src, name))
        return self

    def vel_u16(self) -> torch.Tensor:
        """Velocity codes [n, 3] as int64 values 0..65535 (or 0..255)."""
        v = self.vel[:, :3].to(torch.int64)
        return v & 0xFFFF if self.vel.dtype == torch.int16 else v


def config_struct(cfg: Dict) -> pm_config_t:
    c = pm_config_t()
    c.n_fine = int(cfg["n_fine"])
    c.coarse_ratio = int(cfg.get("coarse_ratio", 1))
    c.tile = int(cfg.get("tile", cfg["n_fine"]))
    c.buffer = int(cfg.get("buffer", 0))
    c.cmp_ratio = int(cfg.get("cmp_ratio", 4))
    c.vel_bits = int(cfg.get("vel_bits", 16))
    c.deposit_mode = int(cfg.get("deposit_mode", 0))
    c.tile_batch = int(cfg.get("tile_batch", 0))
    c.vmax_mode = int(cfg.get("vmax_mode", 0))
    c.pp = int(cfg.get("pp", 0))
    c.G = float(cfg["G"])
    c.mass[0], c.mass[1] = (float(m) for m in cfg["mass"])
    cnt = cfg.get("count", (0, 0))
    c.count[0], c.count[1] = (int(k) for k in cnt)
    c.r_split = float(cfg.get("r_split", 0.0))
    c.r_cut = float(cfg.get("r_cut", 0.0))
    c.r_soft = float(cfg.get("r_soft", 0.0))
    return c


class PM:
    """Handle around pm_init / pm_destroy with one method per entry point."""

    def __init__(self, cfg: Dict):
        self.lib = _lib.load()
        self.cfg = dict(cfg)
        self._cs = config_struct(cfg)
        h = ctypes.c_void_p()
        rc = self.lib.pm_init(ctypes.byref(self._cs), ctypes.byref(h))
        if rc != _lib.PM_OK:
            raise PMError(rc, "pm_init failed")
        self.h = h
        g = [ctypes.c_int64() for _ in range(4)]
        self.lib.pm_geometry(self.h, *[ctypes.byref(x) for x in g])
        self.n_cmp, self.n_coarse, self.n_tiles, self.tile_edge = (int(x.value) for x in g)
        self.n_fine = int(cfg["n_fine"])
        self.two_level = int(cfg.get("coarse_ratio", 1)) > 1
        self.vel_bits = int(cfg.get("vel_bits", 16))

    def close(self):
        if getattr(self, "h", None):
            self.lib.pm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _err(self, rc: int):
        if rc != _lib.PM_OK:
            buf = ctypes.create_string_buffer(512)
            self.lib.pm_last_error(self.h, buf, 512)
            raise PMError(rc, buf.value.decode())

    # ---- entry points -------------------------------------------------
    def check(self, stream=None):
        self._err(self.lib.pm_check(self.h, _stream(stream)))

    def wait_probe(self, limit_cycles: int, stream=None):
        """pm_wait_probe: a device wait that runs out; the next check() raises PM_ERR_TIMEOUT."""
        self._err(self.lib.pm_wait_probe(self.h, int(limit_cycles), _stream(stream)))

    def empty_codes(self, n: int, esc_cap: Optional[int] = None) -> Codes:
        return Codes.empty(n, self.n_cmp, self.vel_bits, esc_cap)

    def decompress(self, species: int, codes: Codes, stream=None) -> Tuple[torch.Tensor, torch.Tensor]:
        x = torch.empty((codes.n, 3), dtype=torch.float32, device="cuda")
        v = torch.empty((codes.n, 3), dtype=torch.float32, device="cuda")
        cs = codes.struct()
        self._err(self.lib.pm_decompress(self.h, species, ctypes.byref(cs), _ptr(x), _ptr(v), _stream(stream)))
        return x, v

    def compress(self, species: int, x: torch.Tensor, v: torch.Tensor, vmax: Optional[torch.Tensor] = None,
                 out: Optional[Codes] = None, stream=None) -> Codes:
        n = x.shape[0]
        out = out if out is not None else self.empty_codes(n)
        cs = out.struct()
        self._err(self.lib.pm_compress(self.h, species, _ptr(x.contiguous()), _ptr(v.contiguous()), _ptr(vmax),
                                       ctypes.byref(cs), _stream(stream)))
        return out

    def zeros_meshes(self, fixed: bool = False):
        dt = torch.int64 if fixed else torch.float32
        rf = torch.zeros((self.n_fine,) * 3, dtype=dt, device="cuda")
        rc = torch.zeros((self.n_coarse,) * 3, dtype=dt, device="cuda") if self.two_level else None
        return rc, rf

    def deposit(self, species: int, x: torch.Tensor, rho_coarse, rho_fine, stream=None):
        self._err(self.lib.pm_deposit(self.h, species, _ptr(x), x.shape[0], _ptr(rho_coarse), _ptr(rho_fine),
                                      _stream(stream)))

    def deposit_weights(self, x: torch.Tensor, w: torch.Tensor, stream=None) -> torch.Tensor:
        """CIC deposit of per-particle weights w [n, nw] (nw <= 4) onto nw fine meshes [nw, n^3]."""
        w = w.reshape(x.shape[0], -1).to(torch.float32).contiguous()
        out = torch.zeros((w.shape[1],) + (self.n_fine,) * 3, dtype=torch.float32, device="cuda")
        self._err(self.lib.pm_deposit_weights(self.h, _ptr(x.contiguous()), x.shape[0], _ptr(w), w.shape[1],
                                              _ptr(out), _stream(stream)))
        return out

    def deposit_fixed(self, species: int, x: torch.Tensor, rho_coarse, rho_fine, stream=None):
        self._err(self.lib.pm_deposit_fixed(self.h, species, _ptr(x), x.shape[0], _ptr(rho_coarse),
                                            _ptr(rho_fine), _stream(stream)))

    def deposit_codes(self, codes: Sequence[Codes], rho_coarse, rho_fine, stream=None):
        arr = (pm_codes_t * 2)(codes[0].struct(), codes[1].struct())
        self._err(self.lib.pm_deposit_codes(self.h, arr, _ptr(rho_coarse), _ptr(rho_fine), _stream(stream)))

    def tile_density(self, rho_fine: torch.Tensor, tile: int, stream=None) -> torch.Tensor:
        T = self.tile_edge
        out = torch.empty((T, T, T), dtype=torch.float32, device="cuda")
        self._err(self.lib.pm_tile_density(self.h, _ptr(rho_fine), tile, _ptr(out), _stream(stream)))
        return out

    def zeros_acc(self):
        af = torch.zeros((3,) + (self.n_fine,) * 3, dtype=torch.float32, device="cuda")
        ac = torch.zeros((3,) + (self.n_coarse,) * 3, dtype=torch.float32, device="cuda") if self.two_level else None
        return ac, af

    def solve(self, rho_coarse, rho_fine, acc_coarse, acc_fine, stream=None):
        fn = self.lib.pm_solve_fixed if rho_fine.dtype == torch.int64 else self.lib.pm_solve
        self._err(fn(self.h, _ptr(rho_coarse), _ptr(rho_fine), _ptr(acc_coarse), _ptr(acc_fine), _stream(stream)))

    def interpolate(self, x: torch.Tensor, acc_coarse, acc_fine, stream=None) -> torch.Tensor:
        a = torch.empty_like(x)
        self._err(self.lib.pm_interpolate(self.h, _ptr(x), x.shape[0], _ptr(acc_coarse), _ptr(acc_fine), _ptr(a),
                                          _stream(stream)))
        return a

    def kick_drift(self, x, v, acc_coarse, acc_fine, c_kick: float, c_drift: float, stream=None):
        self._err(self.lib.pm_kick_drift(self.h, _ptr(x), _ptr(v), x.shape[0], _ptr(acc_coarse), _ptr(acc_fine),
                                         c_kick, c_drift, _stream(stream)))

    def step(self, codes_in: Sequence[Codes], codes_out: Sequence[Codes], c_kick: float, c_drift: float,
             stream=None):
        arr_in = (pm_codes_t * 2)(codes_in[0].struct(), codes_in[1].struct())
        arr_out = (pm_codes_t * 2)(codes_out[0].struct(), codes_out[1].struct())
        self._err(self.lib.pm_step(self.h, arr_in, arr_out, c_kick, c_drift, _stream(stream)))

    def step_host(self, codes_in: Sequence[Codes], codes_out: Sequence[Codes], c_kick: float, c_drift: float,
                  stream=None):
        arr_in = (pm_codes_t * 2)(codes_in[0].struct(), codes_in[1].struct())
        arr_out = (pm_codes_t * 2)(codes_out[0].struct(), codes_out[1].struct())
        self._err(self.lib.pm_step_host(self.h, arr_in, arr_out, c_kick, c_drift, _stream(stream)))

    # ---- uncompressed step and its reverse mode (single periodic mesh) -------
    def density(self, xs: Sequence[torch.Tensor], fixed: bool, stream=None):
        """Deposit both species; returns the mesh (int64 in 2^-32 mass units if fixed)."""
        rc, rf = self.zeros_meshes(fixed=fixed)
        for s, x in enumerate(xs):
            (self.deposit_fixed if fixed else self.deposit)(s, x, rc, rf, stream)
        return rc, rf

    def step_plain(self, xs: Sequence[torch.Tensor], vs: Sequence[torch.Tensor], c_kick: float, c_drift: float,
                   fixed: bool = True, stream=None):
        """One uncompressed step in place: deposit, solve, interpolate + kick + drift.
        Returns the step's fine acceleration mesh [3][n^3] (at the pre-step positions)."""
        rc, rf = self.density(xs, fixed, stream)
        ac, af = self.zeros_acc()
        self.solve(rc, rf, ac, af, stream)
        for x, v in zip(xs, vs):
            self.kick_drift(x, v, ac, af, c_kick, c_drift, stream)
        return af

    def deposit_adjoint(self, species: int, x: torch.Tensor, lam_rho: torch.Tensor, lam_x: torch.Tensor, stream=None):
        self._err(self.lib.pm_deposit_adjoint(self.h, species, _ptr(x), x.shape[0], _ptr(lam_rho), _ptr(lam_x),
                                              _stream(stream)))

    def solve_adjoint(self, lam_acc: torch.Tensor, lam_rho: torch.Tensor, stream=None):
        self._err(self.lib.pm_solve_adjoint(self.h, _ptr(lam_acc), _ptr(lam_rho), _stream(stream)))

    def interpolate_adjoint(self, x, acc, c_kick, c_drift, lam_x, lam_v, lam_acc, stream=None):
        self._err(self.lib.pm_interpolate_adjoint(self.h, _ptr(x), x.shape[0], _ptr(acc), c_kick, c_drift,
                                                  _ptr(lam_x), _ptr(lam_v), _ptr(lam_acc), _stream(stream)))

    def step_adjoint(self, xs: Sequence[torch.Tensor], lam_x: Sequence[torch.Tensor], lam_v: Sequence[torch.Tensor],
                     c_kick: float, c_drift: float, acc_fine: Optional[torch.Tensor] = None, stream=None):
        """Reverse step in place; acc_fine (the step's [3][n^3] acceleration mesh at
        xs) skips its recompute."""
        st = (pm_particles_t * 2)(*[pm_particles_t(x.shape[0], x.data_ptr(), 0) for x in xs])
        lam = (pm_particles_t * 2)(*[pm_particles_t(a.shape[0], a.data_ptr(), b.data_ptr())
                                     for a, b in zip(lam_x, lam_v)])
        if acc_fine is None:
            self._err(self.lib.pm_step_adjoint(self.h, st, lam, c_kick, c_drift, _stream(stream)))
        else:
            self._err(self.lib.pm_step_adjoint_acc(self.h, st, lam, _ptr(acc_fine), c_kick, c_drift,
                                                   _stream(stream)))

    def restrict(self, rho_fine: torch.Tensor, stream=None) -> torch.Tensor:
        """Coarse density from a fine one (CIC restriction)."""
        out = torch.empty((self.n_coarse,) * 3, dtype=torch.float32, device="cuda")
        self._err(self.lib.pm_restrict(self.h, _ptr(rho_fine), _ptr(out), _stream(stream)))
        return out

    def pp_accel(self, codes: Sequence[Codes], stream=None) -> torch.Tensor:
        """Eq. 4 accelerations [n0 + n1, 4] (x, y, z, 0), stream order, species 0 first."""
        acc = torch.empty((codes[0].n + codes[1].n, 4), dtype=torch.float32, device="cuda")
        arr = (pm_codes_t * 2)(codes[0].struct(), codes[1].struct())
        self._err(self.lib.pm_pp_accel(self.h, arr, _ptr(acc), _stream(stream)))
        return acc

    def checkpoint_begin(self, codes: Sequence[Codes], host: Sequence[Codes], stream=None):
        """Queue device -> host copies of both species' codes (host: pinned Codes, same shapes)."""
        dev = (pm_codes_t * 2)(codes[0].struct(), codes[1].struct())
        hst = (pm_codes_t * 2)(host[0].struct(), host[1].struct())
        self._err(self.lib.pm_checkpoint_begin(self.h, dev, hst, _stream(stream)))

    def checkpoint_fence(self, stream=None):
        """Make `stream` wait for the pending checkpoint copies."""
        self._err(self.lib.pm_checkpoint_fence(self.h, _stream(stream)))

    def checkpoint_wait(self):
        """Block until the pending checkpoint copies are in host memory."""
        self._err(self.lib.pm_checkpoint_wait(self.h))

    def pack(self, codes: Codes, stream=None) -> Codes:
        """Packed copy (record bytes, no padding) of device codes."""
        out = Codes.empty_packed(codes.n, self.n_cmp, self.vel_bits, codes.esc.shape[0])
        a, b = codes.struct(), out.struct()
        self._err(self.lib.pm_pack_codes(self.h, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
        return out

    def unpack(self, packed: Codes, stream=None) -> Codes:
        out = Codes.empty(packed.n, self.n_cmp, self.vel_bits, packed.esc.shape[0])
        a, b = packed.struct(), out.struct()
        self._err(self.lib.pm_unpack_codes(self.h, ctypes.byref(a), ctypes.byref(b), _stream(stream)))
        return out

    def step_packed(self, codes_in: Sequence[Codes], codes_out: Sequence[Codes], c_kick: float, c_drift: float,
                    stream=None):
        """pm_step_packed: packed host codes in and out."""
        arr_in = (pm_codes_t * 2)(codes_in[0].struct(), codes_in[1].struct())
        arr_out = (pm_codes_t * 2)(codes_out[0].struct(), codes_out[1].struct())
        self._err(self.lib.pm_step_packed(self.h, arr_in, arr_out, c_kick, c_drift, _stream(stream)))

    def step_packed_async(self, codes_in: Sequence[Codes], codes_out: Sequence[Codes], c_kick: float,
                          c_drift: float, stream=None):
        """pm_step_packed_async: queues copies and step; out is complete after check()."""
        arr_in = (pm_codes_t * 2)(codes_in[0].struct(), codes_in[1].struct())
        arr_out = (pm_codes_t * 2)(codes_out[0].struct(), codes_out[1].struct())
        self._err(self.lib.pm_step_packed_async(self.h, arr_in, arr_out, c_kick, c_drift, _stream(stream)))

    def set_timing(self, on: bool):
        self._err(self.lib.pm_set_timing(self.h, 1 if on else 0))

    @staticmethod
    def _tuning_dict(t: pm_tuning_t) -> Dict:
        return {"deposit_block": tuple(t.deposit_block), "deposit_persistent": t.deposit_persistent,
                "kick_block": tuple(t.kick_block), "kick_window": t.kick_window,
                "kick_persistent": t.kick_persistent, "tile_batch": t.tile_batch}

    def get_tuning(self) -> Dict:
        t = pm_tuning_t()
        self._err(self.lib.pm_get_tuning(self.h, ctypes.byref(t)))
        return self._tuning_dict(t)

    def set_tuning(self, tuning: Dict):
        t = pm_tuning_t()
        self.lib.pm_get_tuning(self.h, ctypes.byref(t))
        for k, v in tuning.items():
            if k in ("deposit_block", "kick_block"):
                getattr(t, k)[:] = [int(a) for a in v]
            else:
                setattr(t, k, int(v))
        self._err(self.lib.pm_set_tuning(self.h, ctypes.byref(t)))

    def autotune(self, codes_in: Sequence[Codes], codes_out: Sequence[Codes], c_kick: float, c_drift: float,
                 reps: int = 2, stream=None) -> Dict:
        """Time candidate launch tunings of step(codes_in -> codes_out) and keep the fastest."""
        arr_in = (pm_codes_t * 2)(codes_in[0].struct(), codes_in[1].struct())
        arr_out = (pm_codes_t * 2)(codes_out[0].struct(), codes_out[1].struct())
        t = pm_tuning_t()
        self._err(self.lib.pm_autotune(self.h, arr_in, arr_out, c_kick, c_drift, reps, _stream(stream),
                                       ctypes.byref(t)))
        return self._tuning_dict(t)

    def set_graphs(self, on: bool):
        """Replay step() as captured CUDA graphs (one per codes/c_k/c_d set)."""
        self._err(self.lib.pm_set_graphs(self.h, 1 if on else 0))

    def stage_times(self) -> Dict[str, Tuple[float, int]]:
        ms = (ctypes.c_float * 64)()
        n = ctypes.c_int()
        names = ctypes.create_string_buffer(4096)
        self._err(self.lib.pm_stage_times(self.h, ms, 64, ctypes.byref(n), names, 4096))
        out = {}
        for i, item in enumerate(names.value.decode().split(";") if n.value else []):
            name, cnt = item.split("#")
            out[name] = (float(ms[i]), int(cnt))
        return out


def serialize(codes_host: Codes, n_cmp: int, vel_bits: int) -> bytes:
    """Sec. 2.4 byte stream of host codes (pm_serialize)."""
    lib = _lib.load()
    cs = codes_host.struct()
    ln = ctypes.c_size_t()
    rc = lib.pm_serialize(ctypes.byref(cs), n_cmp, vel_bits, None, 0, ctypes.byref(ln))
    if rc != _lib.PM_OK:
        raise PMError(rc, "pm_serialize (size)")
    buf = (ctypes.c_uint8 * ln.value)()
    rc = lib.pm_serialize(ctypes.byref(cs), n_cmp, vel_bits, buf, ln.value, ctypes.byref(ln))
    if rc != _lib.PM_OK:
        raise PMError(rc, "pm_serialize")
    return bytes(buf)


def deserialize(data: bytes, n: int, n_cmp: int, vel_bits: int, esc_cap: int = 1024) -> Codes:
    lib = _lib.load()
    out = Codes.empty(n, n_cmp, vel_bits, esc_cap, device="cpu")
    cs = out.struct()
    buf = (ctypes.c_uint8 * len(data)).from_buffer_copy(data)
    rc = lib.pm_deserialize(buf, len(data), n_cmp, vel_bits, ctypes.byref(cs))
    if rc != _lib.PM_OK:
        raise PMError(rc, "pm_deserialize")
    return out
