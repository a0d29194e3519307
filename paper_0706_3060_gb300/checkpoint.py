"""Save and resume a leapfrog run: the device state (positions with masses,
velocities, the acceleration carried into the next step, the optional low
parts of the two-float state), the step count and the run's parameters, in one
``.npz`` file. Resuming continues bit for bit: ``nbody_step`` with
``acc_valid=True`` on the restored state equals the uninterrupted run.

Host-side marshalling only (numpy and torch copies); no arithmetic."""
from __future__ import annotations

import json

import numpy as np
import torch

_FORMAT = 1


def save_state(path, pos_m, vel, acc, *, step: int, params: dict | None = None,
               state_lo=None) -> None:
    """Write the run state to ``path`` (.npz). ``params`` is any JSON-serialisable
    dict (dt, eps, law, ...) stored beside the arrays."""
    arrays = {"pos_m": pos_m.detach().cpu().numpy(), "vel": vel.detach().cpu().numpy(),
              "acc": acc.detach().cpu().numpy()}
    if state_lo is not None:
        arrays["state_lo"] = state_lo.detach().cpu().numpy()
    meta = {"format": _FORMAT, "step": int(step), "params": params or {}}
    np.savez(path, meta=np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8), **arrays)


def load_state(path, device=None) -> dict:
    """Read a state written by save_state; arrays come back as contiguous float32
    tensors on ``device`` (default: the current CUDA device)."""
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device())
    with np.load(path) as z:
        meta = json.loads(bytes(z["meta"]).decode())
        if meta.get("format") != _FORMAT:
            raise ValueError(f"{path}: unknown state format {meta.get('format')}")
        out = {k: torch.from_numpy(np.ascontiguousarray(z[k], dtype=np.float32)).to(device)
               for k in ("pos_m", "vel", "acc", "state_lo") if k in z.files}
    out["step"] = meta["step"]
    out["params"] = meta["params"]
    return out
