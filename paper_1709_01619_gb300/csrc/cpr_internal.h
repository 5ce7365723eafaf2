// cpr_internal.h -- helpers shared by the translation units of the C ABI.
#pragma once

#include "../../include/cpr.h"
#include "cpr_launch.h"

// nullptr when *c is a valid configuration, else a message.
const char* cpr_validate_config(const cpr_config* c);

// Launch description (sizes, spacing, physics, FP64 tables) of a validated
// configuration; false if the tables cannot be built.
bool cpr_fill_launch_cfg(const cpr_config* cfg, cpr::LaunchCfg* out);
